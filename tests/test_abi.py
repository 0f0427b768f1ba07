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


def test_deserialize_rejects_bad_images_without_gpu(librb, oracle_mod):
    """rb_deserialize checks the whole image on the host before any device
    work: images composed from the oracle's layout (the documented format),
    each with one field broken, are refused with RB_EINVAL."""
    import struct
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    from layout_tools import image_from_layout
    vals = np.concatenate([np.arange(0, 62000, 62), np.arange(2**16, 2**16 + 100), np.arange(2**16 + 101, 2**16 + 201),
                           np.arange(2 * 2**16, 3 * 2**16, 2)]).astype(np.uint32)
    lay = oracle_mod.Bitmap.from_sorted(vals).layout()
    img = image_from_layout(lay)
    n = len(lay["keys"])
    keys_at, runs_at, types_at = 32, 32 + 2 * n, 32 + 4 * n
    cards_at = 32 + ((5 * n + 3) // 4) * 4
    meta = cards_at + 4 * n
    bad = {
        "magic": b"XXXX" + img[4:],
        "version": img[:4] + struct.pack("<I", 2) + img[8:],
        "truncated": img[:-1],
        "long": img + b"\0",
        "keys_order": img[:keys_at] + struct.pack("<HH", 1, 0) + img[keys_at + 4:],
        "type_out_of_range": img[:types_at] + bytes([3]) + img[types_at + 1:],
        "card_mismatch": img[:cards_at] + struct.pack("<I", int(lay["cards"][0]) + 1) + img[cards_at + 4:],
        "header_card": img[:16] + struct.pack("<Q", int(lay["cards"].sum()) + 1) + img[24:],
        "array_unsorted": img[:meta] + img[meta + 2:meta + 4] + img[meta:meta + 2] + img[meta + 4:],
        # the run chunk (2 runs) claimed as 1 run, or as 3
        "run_count_low": img[:runs_at + 2] + struct.pack("<H", 1) + img[runs_at + 4:],
        "run_count_high": img[:runs_at + 2] + struct.pack("<H", 3) + img[runs_at + 4:],
        # the runs made adjacent: [2^16, 2^16 + 100) then [2^16 + 100, ...)
        "runs_not_maximal": img[:meta + 2000 + 4] + struct.pack("<H", 100) + img[meta + 2000 + 6:],
        # an array chunk retyped as runs: not canonical and the wrong size
        "retyped": img[:types_at] + bytes([2]) + img[types_at + 1:],
        "empty": b"",
    }
    librb.rb_deserialize.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    for name, data in bad.items():
        out = ctypes.c_void_p()
        assert librb.rb_deserialize(data, len(data), None, ctypes.byref(out)) == 1, name
        assert out.value is None, name
    # a non-canonical but well-formed array: the first chunk's 1000 values
    # replaced by 4097 consecutive ones as an array (canonically runs)
    arr = np.arange(4097, dtype=np.uint16)
    lay2 = {"keys": np.array([0], np.uint16), "types": np.array([0], np.uint8),
            "cards": np.array([4097], np.uint32), "offs": np.array([0, 8194], np.uint64),
            "payload": arr.view(np.uint8)}
    data = image_from_layout(lay2)
    out = ctypes.c_void_p()
    assert librb.rb_deserialize(data, len(data), None, ctypes.byref(out)) == 1


def test_accumulator_argument_checks_without_gpu(librb):
    librb.rb_accum_create.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert librb.rb_accum_create(3, 100, None, ctypes.byref(out)) == 1       # XOR does not accumulate
    assert librb.rb_accum_create(1, 0, None, ctypes.byref(out)) == 1         # no tiles
    assert librb.rb_accum_create(1, 65537, None, ctypes.byref(out)) == 1     # more tiles than keys
    assert librb.rb_accum_create(1, 10, None, None) == 1
    assert out.value is None


def test_binding_rejects_values_outside_u32_without_gpu(librb):
    """The binding narrows user values to uint32 only when they fit: out-of-range
    or non-integer values raise before any device work, and a value outside
    [0, 2^32) is never reported as a member (it would otherwise wrap)."""
    import numpy as np
    import paper_1709_07821_gb300 as rb
    for bad in (np.array([-1, 5]), np.array([1, 2 ** 32], dtype=np.int64), np.array([3, 2 ** 40], dtype=np.uint64)):
        with pytest.raises(ValueError):
            rb.Bitmap.from_sorted(bad)
    with pytest.raises(TypeError):
        rb.Bitmap.from_sorted(np.array([1.0, 2.5]))
    with pytest.raises(ValueError):
        rb._queries([0], [2 ** 32 + 3], [1])
    with pytest.raises(ValueError):
        rb._queries([0], [1], [-2])
    with pytest.raises(ValueError):
        rb.batch_jaccard([], [1], [1, 2])
    unbound = rb.Bitmap(None)            # no device bitmap: these answers need none
    assert (2 ** 32 + 5) not in unbound and -1 not in unbound
    got = unbound.contains(np.array([-1, 2 ** 32, 2 ** 40], dtype=np.int64))
    assert got.dtype == np.uint8 and got.tolist() == [0, 0, 0]
    with pytest.raises(TypeError):
        unbound.contains(np.array([0.5]))
    # in-range inputs pass through unchanged, without a copy for uint32
    v = np.array([0, 7, 2 ** 32 - 1], dtype=np.uint32)
    assert rb._u32(v, "v") is v
    assert rb._u32(np.array([0, 2 ** 32 - 1], dtype=np.int64), "v").tolist() == [0, 2 ** 32 - 1]
    assert rb._u32([], "v").dtype == np.uint32
