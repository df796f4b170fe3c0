"""The reference arm of bench.py (the oracle on the host cores) under a
two-rank torchrun launch: rank 0 alone prints one JSON line, with the keys
the benchmark contract names; the other rank exits 0 without work.  CPU
only; a short oracle budget."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3", "--ref-seconds", "2"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    for key in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_cpu_baseline_fields():
    """The CPU baseline beside the GPU line: the oracle on all cores and on
    one, with window-cells/s, Gbp/s, the core count and the host CPU."""
    sys.path.insert(0, ROOT)
    import bench
    pats = bench.genome_patterns()
    d = bench.cpu_baseline(300_000, pats, 0.2)
    assert d["kind"] == "oracle" and d["unit"] == "window-cells/s" and d["cores"] >= 1
    assert d["value"] > 0 and d["gbp_per_s"] > 0 and d["cpu"]
    one = d["single_thread"]
    assert one["value"] > 0 and one["gbp_per_s"] > 0
    # window-cells per symbol searched: the nine searches' mean pattern length
    ents = bench.entries(pats)
    mean_m = sum(len(p) for p, _ in ents) / len(ents)
    assert abs(d["value"] / (d["gbp_per_s"] * 1e9) - mean_m) < 0.01 * mean_m
