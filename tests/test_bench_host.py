"""Host-side logic of bench.py on CPU: clock parsing, throughput arithmetic,
the max-over-ranks reduction with two gloo ranks, the reporting of a failed
secondary measurement, and the reference arm under torchrun with two ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSV = """index, clocks.current.sm [MHz], clocks.max.sm [MHz], power.draw [W], clocks_event_reasons.active, clocks_event_reasons.hw_slowdown, clocks_event_reasons.hw_thermal_slowdown, clocks_event_reasons.sw_thermal_slowdown, clocks_event_reasons.sw_power_cap
0, 345 MHz, 2070 MHz, 180.00 W, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active
0, 1965 MHz, 2070 MHz, 800.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
0, 1980 MHz, 2070 MHz, 820.00 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active
0, 1950 MHz, 2070 MHz, 810.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
"""


def test_parse_clocks():
    r = bench.parse_clocks(CSV)
    assert r["sm_mhz"] == 1965.0
    assert r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["samples"] == 4
    assert bench.parse_clocks("garbage\n") is None


def test_throughput_and_percentiles():
    assert bench.throughput(3e6, 1.5) == 2e6
    assert bench.percentile([1, 2, 3, 4], 50) == 2.5


def test_reference_arm_rejects_short_warmup():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2"])


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q.put((rank, bench.max_over_ranks(float(rank) + 0.5, world)))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 1.5, 1: 1.5}
    assert bench.max_over_ranks(2.5, 1) == 2.5


def test_secondary_reports_a_failure_in_its_place():
    assert bench.secondary("ok", lambda: {"value": 1}) == {"value": 1}

    def boom():
        raise RuntimeError("device status 8")

    got = bench.secondary("batch", boom)
    assert set(got) == {"error"} and "batch failed" in got["error"] and "status 8" in got["error"]


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched as the scaling run launches it: rank
    0 alone times the oracle and prints one JSON line; rank 1 exits 0 without
    work (no GPU needed)."""
    import json
    import subprocess

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
