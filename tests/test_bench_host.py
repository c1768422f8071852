"""Host-side logic of bench.py (CPU): the DRAM-traffic counters of the render kernel are
reported only while the kernel's sources are the ones they were taken from, and editing a
comment does not count as a change; the reference arm's line keeps its contract."""
import importlib.util
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_strip_comments_keeps_code_only(bench):
    src = "int a = 1; // one\n/* block\n comment */ int b = 2;\n\n   \nint c = a / b;  /* x */\n"
    assert bench._strip_comments(src) == "int a = 1;\n int b = 2;\nint c = a / b;"


def _copy_tree(bench, dst):
    for rel in bench.KERNEL_SOURCES + ["profiles/render_mixed_traffic.txt"]:
        os.makedirs(os.path.join(dst, os.path.dirname(rel)), exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), os.path.join(dst, rel))


def test_traffic_follows_the_kernel_sources(bench, tmp_path, monkeypatch):
    _copy_tree(bench, str(tmp_path))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.kernel_source_hash()
    recorded = bench._load_traffic()  # None when the committed counters are stale
    rel = bench.KERNEL_SOURCES[0]
    path = os.path.join(str(tmp_path), rel)
    with open(path, "a", encoding="utf-8") as f:  # a comment: same code, same counters
        f.write("\n// a note\n/* another */\n")
    assert bench.kernel_source_hash() == base
    assert bench._load_traffic() == recorded
    with open(path, "a", encoding="utf-8") as f:  # code: the counters no longer apply
        f.write("\nstatic int e2e_changed_for_the_test = 1;\n")
    assert bench.kernel_source_hash() != base
    assert bench._load_traffic() is None


def test_reference_arm_line(tmp_path):
    # the reference arm (the FP64 oracle on the host cores) prints one JSON line on the
    # headline's own config, names the sample each step renders, and reports that sample's
    # own time per step, consistent with its value
    import json
    import subprocess
    import sys

    env = dict(os.environ, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, cwd=str(tmp_path), env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    spec = importlib.util.spec_from_file_location("bench_cfg", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    w = mod.W.config2()
    assert d["impl"] == "reference"
    assert d["config"] == mod.headline_config(w, w.model.slices[0].K, w.model.n_stamps, 1, False)
    assert d["metric"] == mod.METRIC and d["unit"] == mod.UNIT and d["higher_is_better"] is True
    assert d["sample"] == d["cpu_baseline"]["sample"] and "order-slices" in d["sample"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(d["stamps_per_step"] / d["value"] * 1e3 - d["ms_per_step"]) <= 1e-6 * d["ms_per_step"]
