"""The benchmark's multi-process aggregation on CPU: two gloo ranks (world size 2, 127.0.0.1)
agree on the slowest rank's time, and the whole-job rate counts every rank's units."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    rate = bench.whole_job_rate(1000, 4, world, ms)
    q.put((rank, ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo_world_2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]           # both ranks see the slowest time
    assert res[0][2] == pytest.approx(1000 * 4 * 2 / 15e-3)  # units of both ranks over that time


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.whole_job_rate(10, 2, 1, 4.0) == pytest.approx(10 * 2 / 4e-3)


def test_emit_appends_json_lines(tmp_path, capsys):
    import json
    import types
    sys.path.insert(0, ROOT)
    import bench
    path = str(tmp_path / "runs.jsonl")
    for v in (1.0, 2.0):
        bench.emit({"metric": "m", "value": v}, types.SimpleNamespace(results=path))
    bench.emit({"metric": "m", "value": 3.0}, types.SimpleNamespace(results=None))
    out = capsys.readouterr().out.strip().splitlines()
    assert [json.loads(x)["value"] for x in out] == [1.0, 2.0, 3.0]
    assert [json.loads(x)["value"] for x in open(path)] == [1.0, 2.0]


def test_reference_arm_runs_on_cpu():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and prints the
    contract's JSON line (no GPU involved)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-step-s", "0.2"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
