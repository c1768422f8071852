"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and exports every
entry point ``include/e2e_render.h`` declares (no GPU compute)."""
import ctypes
import os
import re

import pytest

from paper_2008_05858_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(?:int|void|const char\*)\s+(e2e_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ["e2e_create", "e2e_destroy", "e2e_load_model", "e2e_load_spectrum", "e2e_render",
                     "e2e_fetch_frame", "e2e_last_error"]:
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_binding_wraps_every_declared_symbol():
    assert set(declared_entry_points()) <= set(binding.exported_symbols())


def test_create_without_a_gpu_fails_loudly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(binding.E2EError) as e:
        binding.e2e_create(0)
    assert e.value.code in (binding.E2E_ECUDA, binding.E2E_EINVAL)
    with pytest.raises(RuntimeError):
        binding.Renderer()


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_cheaper_tail_instantiations_cover_every_tail_variant():
    # the render dispatches to the FAR = true instantiation for every tile variant with tail
    # edges (K >= 3) when the plan sets far_tails; the two variant lists must agree on those
    src = open(os.path.join(ROOT, "paper_2008_05858_gb300", "csrc", "render_mixed.cuh")).read()

    def variants(name):
        i = src.index(f"#define {name}(V)")
        j = src.index("\n\n", i)
        return set((int(k), int(x), int(y)) for k, x, y in re.findall(r"V\((\d+), (\d+), (\d+)\)", src[i:j]))

    base, far = variants("E2E_MIXED_VARIANTS"), variants("E2E_MIXED_FAR_VARIANTS")
    assert far == {v for v in base if v[0] >= 3}
