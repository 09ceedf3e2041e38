"""The JSON line of bench.py's reference arm (the CPU oracle on a bounded sample): the keys
and types the benchmark contract fixes, on a 32^3 sample so that it runs in a second."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--sample-n", "32"], capture_output=True, text=True, env=env, cwd=ROOT,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    line = json.loads(lines[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["n_gpus"] == 1 and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and "32^3" in cb["sample"]
    assert cb["host_nproc"] >= 1 and set(cb["per_pair"]) == {"-2.0,0.0", "-2.0,0.5", "-0.5,0.0", "-0.5,0.5"}
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench.job_step_ms(100.0 + 25.0 * rank, ws)  # the ranks' own step times differ
    q.put((rank, ms, bench.job_value(ms, 4, ws)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_the_whole_job_value():
    """Replicas only: with two gloo ranks on the CPU, every rank sees the maximum step time,
    and the whole-job value divides it by all ranks' solves."""
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [125.0, 125.0]
    assert [g[2] for g in got] == [125.0 / 8, 125.0 / 8]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--sample-n", "32"], capture_output=True, text=True, env=env, cwd=ROOT,
                         timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_roofline_traffic_follows_the_autotuners_choice():
    """The roofline line's DRAM traffic comes from the capture of the sweep variant the
    autotuner kept, matched on its exact description (the balanced form is not taken for the
    256-thread one, nor the other way round); a variant without a capture gives none."""
    sys.path.insert(0, ROOT)
    import bench
    line = "sweep32 n=512 bg gap coef: tile 64x16 nz 32 pair {} ms (variants tried, ms: 10:0.9370 14:0.9904)"
    assert bench.sweep_capture(line.format("0.937099"))[2] == 111
    assert bench.sweep_capture(line.replace("pair", "pair bal").format("0.99"))[2] == 115
    assert bench.sweep_capture(line.replace("pair", "col").format("0.97"))[2] == 119
    assert bench.sweep_capture(line.replace("nz 32", "nz 64").format("1.1")) is None
