"""Host-side pieces of bench.py: the reference arm (the oracle on the host
cores) prints the contract's JSON line, and the roofline helpers compute
what they state."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_roofline_helpers():
    b = _bench_module()
    W = dict(b.WORKLOAD)
    rb = b._roofline_bytes(W)
    # n = 10^6, d = 128, N = 8192, L = 3: 123 blocks, 3194 B per query-point
    assert rb["K"] == 123 and rb["total"] == 3_194_093_568
    tr = b._mac_traffic(rb, W)
    assert 0.98 < tr / rb["total"] < 1.0            # the capture's DRAM bytes scaled by blocks
    assert b._mac_traffic(rb, dict(W, d=96)) is None  # another shape: no scaled figure
    # the batched GEMM at 64 queries, n = 10^7 (K = 1221), d = 96, L = 3
    assert abs(b._batched_flops(64, 1221, 96, 3, 8192) - 4.72e13) < 0.005e13
    assert b._batched_flops(1, 1, 90, 1, 64) == 2.0 * 16 * 1 * (8 * 96) * 1 * 64
    rep = b._ntt_report(738, 8192, 0.5, "x")
    assert abs(rep["polys_per_s"] - 738 / 0.5e-3) < 1e-6
    assert abs(rep["hbm_gbs"] - 16 * 8192 * 738 / 0.5e-3 / 1e9) < 1e-9


def test_all_cores_baseline_uses_every_core():
    b = _bench_module()
    r = b.cpu_baseline_all_cores(quick=True)
    assert r["kind"] == "oracle" and r["value"] > 0
    assert r["cores"] == max(1, min(len(os.sched_getaffinity(0)), 64))


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun only rank 0 runs and prints the reference line
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
