"""The multi-process path of bench.py on CPU: two gloo ranks launched the way
torchrun launches them (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* in the
environment).  Replicas run independently, so the job's time is the slowest
rank's and the whole-job rate counts the units of every rank; the reference
arm runs on rank 0 only."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, units, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    bench = _bench()
    dist = bench._init_dist("gloo")
    try:
        t_job = bench._max_over_ranks(dist, times[rank], "cpu")
        rate = bench._job_rate(units, world, t_job)
        out.put((rank, t_job, rate, bench._reference_runs_here()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(1.5, 2.0), (3.0, 0.25)])
def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_rank(times):
    world, port, units = 2, _free_port(), 1000.0
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, units, out))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    t_max = max(times)
    for rank, t_job, rate, ref_here in res:
        assert t_job == t_max
        assert rate == pytest.approx(world * units / t_max)
        assert ref_here == (rank == 0)


def test_single_process_needs_no_process_group(monkeypatch):
    for v in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(v, raising=False)
    bench = _bench()
    assert bench._init_dist("gloo") is None
    assert bench._max_over_ranks(None, 2.5, "cpu") == 2.5
    assert bench._job_rate(10.0, 1, 2.0) == 5.0
    assert bench._reference_runs_here()


def test_reference_arm_prints_one_json_line():
    """bench.py --impl reference (the FP64 oracle on host cores) at N = 1."""
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    for v in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        env.pop(v, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 1 and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0
