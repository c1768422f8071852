"""Host-side logic of bench.py (CPU): the DRAM-traffic counters of the render kernel are
reported only while the kernel's sources are the ones they were taken from, and editing a
comment does not count as a change."""
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
