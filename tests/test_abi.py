"""C ABI checks that need no GPU: the library loads and exports every entry
point declared in include/avl.h, and the binding mirrors them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "avl.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(avl_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_03901_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared()
    for must in ("avl_create", "avl_step", "avl_get_f", "avl_get_rho", "avl_get_E",
                 "avl_init_markers", "avl_destroy", "avl_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_header():
    from paper_1804_03901_gb300 import avl
    assert sorted(avl.EXPORTED) == declared()
    for n in declared():
        assert callable(getattr(avl, n))


def test_struct_layouts_match_header():
    """Field offsets of the ctypes mirrors equal the C layout (natural alignment)."""
    from paper_1804_03901_gb300 import avl
    assert ctypes.sizeof(avl.avl_domain) == 40
    assert avl.avl_species.vmin.offset == 32 and ctypes.sizeof(avl.avl_species) == 80
    assert avl.avl_f0.beam_n.offset == 8 and avl.avl_f0.nmode.offset == 232
    assert avl.avl_f0.amp.offset == 496


def test_create_rejects_bad_arguments_without_gpu_work(lib):
    """Argument validation happens before any device call."""
    from paper_1804_03901_gb300 import avl
    dom = avl.make_domain(1, 2, 1.0, 0.1)          # nx < 4
    sp = avl.make_species(-1.0, 1.0, (8,), (-1.0,), (1.0,))
    ctx = ctypes.c_void_p()
    st = avl.avl_create(ctypes.byref(dom), (avl.avl_species * 1)(sp), 1, None, ctypes.byref(ctx))
    assert st == avl.AVL_EINVAL and not ctx.value
    assert b"nx" in avl.avl_last_error(None)
    dom = avl.make_domain(1, 16, 1.0, 0.1)
    bad = avl.make_species(-1.0, 0.0, (8,), (-1.0,), (1.0,))   # zero mass
    st = avl.avl_create(ctypes.byref(dom), (avl.avl_species * 1)(bad), 1, None, ctypes.byref(ctx))
    assert st == avl.AVL_EINVAL
    st = avl.avl_create(ctypes.byref(dom), (avl.avl_species * 1)(sp), 0, None, ctypes.byref(ctx))
    assert st == avl.AVL_EINVAL
