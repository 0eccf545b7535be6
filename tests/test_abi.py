"""The C-ABI library builds, loads and exports every entry point declared in
include/mrsim.h (no compute calls: this runs without a GPU)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mrsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mrsim_[a-z_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_03960_gb300 import build, mrsim
    build.build()
    return mrsim.load_library()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ("mrsim_phantom", "mrsim_sequence", "mrsim_group", "mrsim_run"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2508_03960_gb300 import mrsim
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(mrsim.EXPORTS) == names


def test_calls_without_a_device_fail_cleanly(lib):
    """On a machine without a GPU the library reports an error instead of
    crashing or computing anything elsewhere."""
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.mrsim_create(ctypes.byref(h), 0, None)
    assert rc != 0 and not h.value
    assert lib.mrsim_create(None, 0, None) == 1  # MRSIM_EINVAL


def test_binding_refuses_a_missing_library(tmp_path):
    from paper_2508_03960_gb300 import mrsim
    with pytest.raises(ImportError):
        mrsim.load_library(str(tmp_path / "libmrsim.so"))


def test_binding_constants_equal_the_header():
    """Every integer the Python binding names (status codes, modes, flags,
    types, tuning parameters) has the value of the header's #define."""
    from paper_2508_03960_gb300 import mrsim
    src = open(os.path.join(ROOT, "include", "mrsim.h")).read()
    defines = {m.group(1): int(m.group(2))
               for m in re.finditer(r"^#define MRSIM_([A-Z0-9_]+)\s+(\d+)u?\b", src, flags=re.M)}
    checked = 0
    for name, value in defines.items():
        if hasattr(mrsim, name):
            assert getattr(mrsim, name) == value, name
            checked += 1
    assert checked >= 30
