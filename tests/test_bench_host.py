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

