"""The C-ABI library loads, exports every symbol include/*.h declares, and
rejects bad arguments on the host before touching a GPU (runs without one)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(stencil_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2103_08825_gb300 as sg
    return sg


def test_header_lists_entry_points():
    names = declared_functions()
    assert "stencil_run" in names and "stencil_plan_create" in names and len(names) >= 20


def test_library_exports_every_declared_symbol(built):
    lib = built.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(built.EXPORTS)


def test_status_strings(built):
    lib = built.load()
    assert lib.stencil_status_string(0) == b"ok"
    assert lib.stencil_status_string(5) == b"device-side wait timed out"


@pytest.mark.parametrize("kwargs,code", [
    (dict(dim=4, radius=1, shape=(4, 4, 4, 4), pattern=0, weights=[1.0] * 9), 1),
    (dict(dim=2, radius=0, shape=(4, 4), pattern=0, weights=[1.0]), 1),
    (dict(dim=2, radius=1, shape=(4, 4), pattern=0, weights=[1.0] * 4), 1),
    (dict(dim=2, radius=1, shape=(4, 0), pattern=0, weights=[1.0] * 5), 1),
    (dict(dim=2, radius=1, shape=(4, 4), pattern=1, weights=[1.0] * 5), 1),
    (dict(dim=1, radius=1, shape=(8,), pattern=0, weights=[0.5, 0.25, 0.25], dtype=4), 1),
    (dict(dim=1, radius=1, shape=(8,), pattern=0, weights=[1, 2, 1], dtype=9), 1),
])
def test_invalid_plans_rejected_on_host(built, kwargs, code):
    with pytest.raises(built.StencilError) as e:
        built.stencil_plan_create(**kwargs)
    assert e.value.status == code


def test_integer_boundary_value_must_be_integral(built):
    with pytest.raises(built.StencilError) as e:
        built.stencil_plan_create(1, 1, (8,), 0, [2, 1, 1], 0, 0.5, 4)
    assert e.value.status == 1


def test_no_cpu_fallback_without_library(tmp_path):
    import paper_2103_08825_gb300 as sg
    saved = sg._lib
    sg._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            sg.load(str(tmp_path / "missing.so"))
    finally:
        sg._lib = saved
