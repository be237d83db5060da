"""bench.py's multi-rank aggregation on CPU: two gloo ranks (the GPU runs use
NCCL with the same calls).  Every rank runs the whole workload (weak
scaling); the job's time is the slowest rank's and its throughput is the
units of all ranks over that time."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.reduce_max(times[rank], dist, "cpu")
    v = bench.job_rate(ws, 1000.0, t)
    dist.barrier()
    out.put((rank, t, v))
    dist.destroy_process_group()


@pytest.mark.parametrize("times", [(2.0, 3.0), (5.0, 1.0)])
def test_two_ranks_take_the_slowest_time(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == max(times)
        assert v == pytest.approx(2 * 1000.0 / max(times))


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1.5, None, "cpu") == 1.5
    assert bench.job_rate(1, 10.0, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    """Ranks other than 0 of the reference arm exit without work."""
    sys.path.insert(0, ROOT)
    import bench

    class A:
        n, steps, warmup = 64, 1, 0

    bench.run_reference(A(), 2, 1)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_carries_the_contract_keys(capsys):
    """Rank 0 of the reference arm times the FP64 oracle on a strip of the
    workload and prints one JSON line with the GPU arm's metric, unit and
    workload, its own cpu_baseline, and an e2e with no host-device bytes."""
    import json
    sys.path.insert(0, ROOT)
    import bench

    class A:
        n, steps, warmup = 64, 3, 3

    bench.run_reference(A(), 1, 0)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (3, 3, 1)
    assert d["ms_per_step"] > 0 and d["scaling"] == "weak" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_is_reported_only_for_the_kernel_it_was_measured_on(tmp_path, monkeypatch):
    """bench.py scales the committed ncu DRAM bytes per node to a launch, and
    reports null once the kernel sources differ from the ones the counters
    were taken on (their hash is stored beside the figure)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"kernel_sources_sha": bench.kernel_sources_sha(), "dram_bytes_per_node": 60.0}))
    stale = tmp_path / "stale.json"
    stale.write_text(json.dumps({"kernel_sources_sha": "0" * 16, "dram_bytes_per_node": 60.0}))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", {"SMRT": str(good), "MRT_RAW": str(stale)})
    assert bench.traffic_per_launch(1000, "SMRT") == 60000.0
    assert bench.traffic_per_launch(1000, "MRT_RAW") is None
    assert bench.traffic_per_launch(1000, "SMRT_FNEQ") is None

