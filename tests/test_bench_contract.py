"""The benchmark's command-line contract: one JSON line with the keys the
measurement needs, for the CPU reference arm (the oracle, no GPU needed) and,
on a GPU, for this library's arm; and the algorithmic operation count that
the roofline fraction is computed from."""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
BASE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
             "scaling", "vs_baseline", "dtype", "data", "config", "e2e")


def run_bench(*args, timeout=600, env=None):
    e = dict(os.environ)
    e.pop("WORLD_SIZE", None)
    e.pop("RANK", None)
    if env:
        e.update(env)
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), *args], cwd=ROOT, env=e, timeout=timeout,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    return r


def last_json(out: str) -> dict:
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out[-2000:]
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,sample", [("powder", 20_000), ("batched", 5_000)])
def test_reference_arm_prints_one_contract_line(workload, sample):
    r = run_bench("--impl", "reference", "--workload", workload, "--steps", "2", "--warmup", "1",
                  "--ref-sample", str(sample))
    assert r.returncode == 0, r.stderr[-2000:]
    d = last_json(r.stdout)
    for k in BASE_KEYS:
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "histories/s"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_gpus_must_match_the_launched_ranks():
    r = run_bench("--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", timeout=120)
    assert r.returncode != 0
    assert "WORLD_SIZE" in (r.stderr + r.stdout)


def test_algorithmic_operation_count():
    sys.path.insert(0, str(ROOT))
    import bench
    c = {"histories": 2, "events": 10, "collisions": 1, "crossings": 9}
    assert bench.algorithmic_ops_per_history(c) == (187 * 10 + 40 * 1 + 40 * 9) / 2
    assert (bench.OPS_PER_EVENT, bench.OPS_PER_COLLISION, bench.OPS_PER_CROSSING) == (187, 40, 40)


@pytest.mark.gpu
def test_our_arm_prints_one_contract_line_with_roofline_and_e2e():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = run_bench("--steps", "3", "--warmup", "3", "--histories", "10000000", "--batched-steps", "1",
                  "--no-cpu-baseline", timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = last_json(r.stdout)
    for k in BASE_KEYS + ("roofline", "gpu_launches", "clocks", "peaks", "batched_adjoint"):
        assert k in d, k
    rf = d["roofline"]
    assert rf["bound"] == "alu" and rf["unit"] == "lane-ops/s" and rf["peak"] > 1e12
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) <= 1e-9 * rf["frac"]
    assert 0 < rf["frac"] < 1.5
    assert d["gpu_launches"] >= 3 and d["steps"] == 3
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["batched_adjoint"]["value"] > 0 and d["batched_adjoint"]["gpu_launches_per_step"] >= 2
    assert d["tally"]["counters"]["histories"] == 3 * 10_000_000
