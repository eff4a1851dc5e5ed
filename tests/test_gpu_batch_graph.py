"""lqt_solve_batched as a CUDA graph, batches whose descriptors span several
parameter blocks, and large batches whose state sizes run on forked streams.

The call builds one descriptor per problem on the host and hands them to the
device as kernel parameters (32 000 bytes per launch), so that it never waits
for the stream and can be captured.  600 problems (300 at n = 4, 300 at n = 8)
need several blocks per size; every problem is checked against the FP64 oracle
after an eager call, after a replay of the captured call, and after a replay
with new references written into the same input buffers."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, compare, oracle_solve
from paper_2104_03186_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problems(seed0):
    rng = np.random.default_rng(seed0)
    specs = [(4, int(t)) for t in rng.integers(16, 65, size=300)]
    specs += [(8, int(t)) for t in rng.integers(16, 65, size=300)]
    return [inputs.diag_tracking(n, T=T, seed=seed0 + i).rounded_to(np.float32)
            for i, (n, T) in enumerate(specs)]


def _check(probs, outs):
    for p, o in zip(probs, outs):
        compare({k: v.double().cpu().numpy() for k, v in o.items()}, oracle_solve(p), FP32_TOL)


def test_many_descriptors_eager_and_captured():
    import torch

    from paper_2104_03186_gb300 import lqt

    probs = _problems(4000)
    Ps = [lqt.Problem.from_inputs(p) for p in probs]
    outs = [P.allocate_outputs() for P in Ps]
    ws = torch.empty(lqt.lqt_batch_workspace_bytes(Ps, outs), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    lqt.lqt_solve_batched(Ps, outs, ws, stream)
    assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_OK
    _check(probs, outs)
    eager = [{k: v.clone() for k, v in o.items()} for o in outs]

    # capture on a side stream, then replay into zeroed outputs
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        lqt.lqt_solve_batched(Ps, outs, ws, side)
    stream.wait_stream(side)
    for o in outs:
        for v in o.values():
            v.zero_()
    graph.replay()
    assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_OK
    for o, e in zip(outs, eager):
        for k in o:
            assert torch.equal(o[k], e[k]), k  # same kernels, same inputs: bit for bit

    # new references in the same buffers: the replay solves the new problems
    rng = np.random.default_rng(5)
    for p, P in zip(probs, Ps):
        p.r = rng.standard_normal(p.r.shape).astype(np.float32)
        P.arrays["r"].copy_(torch.from_numpy(p.r).reshape(P.arrays["r"].shape))
    graph.replay()
    assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_OK
    _check(probs, outs)


def test_large_batch_runs_its_sizes_side_by_side():
    """A batch of at least 2^20 steps runs each lane size on its own forked
    stream beside the n = 4 launch.  88 problems of 4096 steps per size
    (1.08M steps in all): the one call, eager and replayed from a CUDA graph,
    must equal per-size calls (each under the threshold, one stream) bit for
    bit, and two problems per size must match the oracle."""
    import torch

    from paper_2104_03186_gb300 import lqt

    specs = [(n, 4096) for n in (4, 8, 16) for _ in range(88)]
    probs = [inputs.diag_tracking(n, T=T, seed=5000 + i).rounded_to(np.float32)
             for i, (n, T) in enumerate(specs)]
    Ps = [lqt.Problem.from_inputs(p) for p in probs]
    assert sum(p.T for p in probs) >= 1 << 20
    stream = torch.cuda.current_stream()

    def call(idx, outs):
        sub = [Ps[i] for i in idx]
        o = [outs[i] for i in idx]
        ws = torch.empty(lqt.lqt_batch_workspace_bytes(sub, o), dtype=torch.uint8, device="cuda")
        lqt.lqt_solve_batched(sub, o, ws, stream)
        assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_OK

    alone = [P.allocate_outputs() for P in Ps]
    for n in (4, 8, 16):
        call([i for i, (m, _) in enumerate(specs) if m == n], alone)
    together = [P.allocate_outputs() for P in Ps]
    call(list(range(len(Ps))), together)
    for a, b in zip(alone, together):
        for k in a:
            assert torch.equal(a[k], b[k]), k

    ws = torch.empty(lqt.lqt_batch_workspace_bytes(Ps, together), dtype=torch.uint8,
                     device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        lqt.lqt_solve_batched(Ps, together, ws, side)
    stream.wait_stream(side)
    for o in together:
        for v in o.values():
            v.zero_()
    graph.replay()
    assert lqt.lqt_workspace_status(ws, stream) == lqt.LQT_OK
    for a, b in zip(alone, together):
        for k in a:
            assert torch.equal(a[k], b[k]), k
    for n in (4, 8, 16):
        for i in [i for i, (m, _) in enumerate(specs) if m == n][:2]:
            compare({k: v.double().cpu().numpy() for k, v in together[i].items()},
                    oracle_solve(probs[i]), FP32_TOL)
