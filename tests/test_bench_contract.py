"""bench.py's reference arm on CPU: one JSON line with the contract's keys, the same metric, unit and
workload as the GPU arm, and the oracle described as the baseline that produced it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    sys.path.insert(0, ROOT)
    import bench
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1 and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith(bench.CONFIG_NAME)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["unit"] == d["unit"]
    assert cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_implicit_summary_reports_chosen_and_lagged_against_plain():
    """The default line's implicit object: the chosen variant's and the lagged variant's speed-ups
    over the plain step come from the variants' own step times, kernels are left out."""
    sys.path.insert(0, ROOT)
    import bench
    res = {"metric": "m", "config": "c", "n_dof": 10, "dt_s": 60.0, "steps": 3,
           "variants": {"plain_bj": {"wall_s_per_step": [6.0, 6.0, 6.0], "kernels_last_step": {"k": 1}},
                        "mixed_bj16": {"wall_s_per_step": [1.0, 1.0, 1.0], "kernels_last_step": {"k": 1}},
                        "mixed_bj16_lag3": {"wall_s_per_step": [1.0, 0.7, 0.7], "kernels_last_step": {"k": 1}}},
           "speedup_mixed_bj16_vs_plain_bj": 6.0, "speedup_mixed_bj16_lag3_vs_plain_bj": 7.5}
    s = bench.implicit_summary(res, "mixed_bj16")
    assert s["chosen"] == "mixed_bj16" and s["speedup_chosen_vs_plain"] == 6.0
    assert s["speedup_lagged_vs_plain"] == 7.5
    assert all("kernels_last_step" not in v for v in s["variants"].values())
    assert "lagged" in bench.IMPLICIT_VARIANTS["mixed_bj16_lag3"]["precond_refresh"]
