"""Host logic of bench.py's multi-GPU form (replicas only): world-size-2
gloo ranks on CPU agree on the slowest rank's time and the whole-job value,
and the reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = bench.reduce_max(times[rank], dist, world, "cpu")
    v = bench.whole_job_value(world, 1000, 10, t)
    out.put((rank, t, v))
    dist.destroy_process_group()


def test_replicas_reduce_to_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.25, 0.4]
    ps = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [0.4, 0.4]
    # 2 ranks x 1000 units x 10 steps in 0.4 s = 0.05 M units/s
    assert all(abs(r[2] - 0.05) < 1e-12 for r in res)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line(tmp_path):
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["H"] == d["config"]["W"] == 2048 and d["config"]["K"] == 16


def test_ncu_counters_only_for_the_sources_they_were_taken_on(monkeypatch, tmp_path):
    """The roofline's `traffic` comes from a stored ncu capture; it is
    reported only for the launch size it was taken (or scaled) to, and only
    while the kernel's code (comments and blank space aside) hashes to the
    capture's value: dropped (null) as soon as the code changes."""
    sys.path.insert(0, ROOT)
    import bench
    entry = bench.NCU_COUNTERS["k_step_tile"]
    current = dict(entry, sha=bench.source_code_hash(entry["sources"]))
    monkeypatch.setitem(bench.NCU_COUNTERS, "k_step_tile", current)
    H, W = entry["size"]
    assert bench.ncu_counters("k_step_tile", H, W) == current
    assert bench.ncu_counters("k_step_tile", H // 2, W) is None   # another launch size
    monkeypatch.setitem(bench.NCU_COUNTERS, "k_step_tile", dict(entry, sha="0" * 16))
    assert bench.ncu_counters("k_step_tile", H, W) is None
    assert bench.ncu_counters("no_such_kernel", H, W) is None
    # a comment or blank-space edit keeps the hash, a code edit changes it
    d = tmp_path / "paper_2604_21984_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f = d / "k.cu"
    f.write_text("int f(int a) {\n  return a + 1;  // one more\n}\n")
    h0 = bench.source_code_hash(["k.cu"])
    f.write_text("/* the successor */\nint f(int a) {\n\n    return a + 1;  // the next integer\n}\n")
    assert bench.source_code_hash(["k.cu"]) == h0
    f.write_text("int f(int a) {\n  return a + 2;  // one more\n}\n")
    assert bench.source_code_hash(["k.cu"]) != h0
