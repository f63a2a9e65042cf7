"""Host-side pieces of the benchmark on CPU: the source hash that ties the
committed ncu counters to the planner kernel ignores comments but not code."""
import os

import bench


def _hash_of(tmp_path, edit):
    csrc = tmp_path / "paper_2503_06757_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("prrtc_device.cuh", "prrtc_launch.h", "prrtc_plan.cu"):
        text = open(os.path.join(bench.ROOT, "paper_2503_06757_gb300", "csrc", f), encoding="utf-8").read()
        (csrc / f).write_text(edit(f, text), encoding="utf-8")
    old = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        return bench.kernel_source_hash()
    finally:
        bench.ROOT = old


def test_source_hash_ignores_comments_but_not_code(tmp_path):
    base = bench.kernel_source_hash()
    commented = _hash_of(tmp_path / "a", lambda f, t: t.replace("\n", "\n// a note\n", 3) + "\n/* block */\n")
    assert commented == base
    changed = _hash_of(tmp_path / "b", lambda f, t: t + "\nstatic const int kAnother = 1;\n" if f == "prrtc_plan.cu"
                       else t)
    assert changed != base



def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints
    one JSON line with the contract's keys, the reference marker and an
    end-to-end figure equal to its own value (no device copies)."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--problems", "12"], capture_output=True, text=True, timeout=600,
                       cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
