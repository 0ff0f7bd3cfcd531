"""bench.py --impl reference on CPU: the oracle arm prints one JSON line in the
same metric and unit as the GPU arm of its workload, with the reference-arm
fields (impl, cpu_baseline describing the run, e2e with no host-device bytes)
and one value throughout."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    env = dict(os.environ)
    env.pop("RANK", None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("args,unit,workload", [
    (("--m", "64", "--steps", "2", "--warmup", "1"), "unit-cell steps/s", "kagome_yc8_l12_m2048"),
    (("--workload", "disorder64", "--steps", "1", "--warmup", "1"), "realisation unit-cell steps/s",
     "disorder64"),
])
def test_reference_arm_line(args, unit, workload):
    import bench
    d = _run(*args)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == unit and d["higher_is_better"] is True and d["config"]["workload"] == workload
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(1e3 * (64 if workload == "disorder64" else 1)
                                                                / d["value"], rel=1e-9)
    cb, e2e = d["cpu_baseline"], d["e2e"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == unit
    assert cb["cores"] >= 1 and cb["sample"]
    assert e2e == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prices_the_settled_count_at_the_bench_size():
    """At the kagome cylinder's own m the step model takes the FP64 path's
    settled Lanczos count, elsewhere the paper's 40."""
    import bench
    assert bench.SETTLED_FP64_ITERS["kagome_yc8_l12_m2048"] > bench.PAPER_LANCZOS_ITERS
    d = _run("--m", "64", "--steps", "1", "--warmup", "0")
    assert "40.0 matvecs, the paper's count" in d["cpu_baseline"]["sample"]
