"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/pic.h declares (no device calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pic.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1606_02862_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    names = _declared()
    assert "pic_create" in names and "pic_step" in names
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_1606_02862_gb300 import pic

    assert sorted(pic.EXPORTED) == _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1606_02862_gb300 import pic

    saved = pic._lib
    pic._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            pic.library(str(tmp_path / "missing.so"))
    finally:
        pic._lib = saved


def test_create_rejects_bad_arguments_without_touching_the_device(libpath):
    """Argument checks run before any CUDA call."""
    from paper_1606_02862_gb300 import pic

    L = pic.library(libpath)
    ctx = ctypes.c_void_p()
    g = (pic.Grid * 1)(pic.Grid(16, 16, 16))
    sp = (pic.SpeciesC * 1)(pic.SpeciesC(-1.0, 1.0, 2, 1))
    dx = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    # dt above half a cell per step: rejected as a CFL violation
    assert L.pic_create(g, 1, dx, 0.6, sp, 1, None, ctypes.byref(ctx)) == 2
    # zero boxes, bad shape, nonpositive mass
    assert L.pic_create(g, 0, dx, 0.2, sp, 1, None, ctypes.byref(ctx)) == 1
    for shape in (0, 4):  # 1 CIC, 2 TSC, 3 PCS
        bad = (pic.SpeciesC * 1)(pic.SpeciesC(-1.0, 1.0, shape, 1))
        assert L.pic_create(g, 1, dx, 0.2, bad, 1, None, ctypes.byref(ctx)) == 1
    bad = (pic.SpeciesC * 1)(pic.SpeciesC(-1.0, 0.0, 2, 1))
    assert L.pic_create(g, 1, dx, 0.2, bad, 1, None, ctypes.byref(ctx)) == 1
    bad = (pic.SpeciesC * 1)(pic.SpeciesC(-1.0, 1.0, 2, 1, 2, 0))  # no gather mode 2
    assert L.pic_create(g, 1, dx, 0.2, bad, 1, None, ctypes.byref(ctx)) == 1
    assert not ctx.value
