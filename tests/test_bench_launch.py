"""bench.py's launch contract on CPU: under torch.distributed.run with two
ranks the reference arm (the oracle) runs on rank 0 alone, prints exactly
one JSON line, and every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_batched_oracle_baseline_on_every_core():
    """The batched workload's CPU baseline: the oracle over every window on a
    thread pool, and on one core over a prefix of the windows; both rates
    positive and the core counts stated."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import workloads as W
    toks, off, _ = W.config3_windows(6, lo=1024, hi=4096)
    r = bench.batched_cpu_baseline(toks, off)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert r["one_core"]["cores"] == 1 and r["one_core"]["value"] > 0
    assert f"all 6 windows ({int(off[-1])} tokens)" in r["sample"]
    assert np.all(np.diff(off.astype(np.int64)) >= 1024)
