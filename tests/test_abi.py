"""The C ABI library loads and exports every entry point include/rb.h
declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "rb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(rb_[a-z0-9_]+)\s*\(", src))
    names -= {"rb_alloc_fn", "rb_free_fn"}
    return sorted(names)


@pytest.fixture(scope="module")
def librb():
    from paper_1709_07821_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_surface():
    names = declared()
    for must in ["rb_from_sorted_u32", "rb_to_u32", "rb_and", "rb_or", "rb_andnot", "rb_xor",
                 "rb_and_cardinality", "rb_jaccard", "rb_batch_op", "rb_multi_op", "rb_export_layout",
                 "rb_free", "rb_last_error", "rb_plan_create", "rb_server_create"]:
        assert must in names


def test_every_declared_symbol_is_exported(librb):
    missing = [n for n in declared() if not hasattr(librb, n)]
    assert not missing, missing


def test_version_and_error_strings(librb):
    librb.rb_version.restype = ctypes.c_char_p
    librb.rb_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in librb.rb_version()
    assert isinstance(librb.rb_last_error(), bytes)


def test_argument_checks_without_gpu(librb):
    # calls that fail on their arguments before touching the device
    librb.rb_cardinality.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert librb.rb_cardinality(None, None) == 1
    librb.rb_from_sorted_u32.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert librb.rb_from_sorted_u32(None, 5, 0, None, ctypes.byref(out)) == 1
    assert out.value is None
    librb.rb_multi_op.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p]
    assert librb.rb_multi_op(2, None, 0, None, None, None) == 1      # ANDNOT is not multi-way
