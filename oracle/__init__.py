"""Python handle on the plain CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check
and by the benchmark's CPU-baseline leg, never by the product library.  It
shares no code with the CUDA path.  See oracle.c for what it computes and the
passages of the paper each step follows.

ctypes releases the GIL during each C call, so independent oracle calls run in
parallel from a thread pool.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

AND, OR, ANDNOT, XOR = 0, 1, 2, 3
ARRAY, BITSET, RUN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain C99, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.orc_from_sorted_u32.restype = vp
        lib.orc_from_sorted_u32.argtypes = [vp, u64, ctypes.POINTER(i32)]
        lib.orc_op.restype = vp
        lib.orc_op.argtypes = [i32, vp, vp]
        lib.orc_op_card.restype = u64
        lib.orc_op_card.argtypes = [i32, vp, vp]
        lib.orc_card.restype = u64
        lib.orc_card.argtypes = [vp]
        lib.orc_jaccard.restype = ctypes.c_double
        lib.orc_jaccard.argtypes = [vp, vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        lib.orc_cosine.restype = ctypes.c_double
        lib.orc_cosine.argtypes = [vp, vp, ctypes.POINTER(u64)]
        lib.orc_contains.argtypes = [vp, vp, u64, vp]
        lib.orc_multi.restype = vp
        lib.orc_multi.argtypes = [i32, ctypes.POINTER(vp), u32]
        lib.orc_n.restype = u32
        lib.orc_n.argtypes = [vp]
        lib.orc_payload_bytes.restype = u64
        lib.orc_payload_bytes.argtypes = [vp]
        lib.orc_to_u32.restype = u64
        lib.orc_to_u32.argtypes = [vp, vp, u64]
        lib.orc_export.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.orc_free.argtypes = [vp]
        _lib = lib
    return _lib


class OracleError(Exception):
    pass


class Bitmap:
    """An oracle Roaring bitmap (host memory, canonical form)."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def from_sorted(cls, values) -> "Bitmap":
        lib = _load()
        v = np.ascontiguousarray(values, dtype=np.uint32)
        st = ctypes.c_int(0)
        h = lib.orc_from_sorted_u32(v.ctypes.data if v.size else None, v.size, ctypes.byref(st))
        if st.value == 1:
            raise ValueError("input must be strictly increasing")
        if not h:
            raise MemoryError("oracle allocation failed")
        return cls(h)

    def op(self, op: int, other: "Bitmap") -> "Bitmap":
        h = _load().orc_op(op, self._h, other._h)
        if not h:
            raise MemoryError("oracle allocation failed")
        return Bitmap(h)

    def op_card(self, op: int, other: "Bitmap") -> int:
        return int(_load().orc_op_card(op, self._h, other._h))

    def jaccard(self, other: "Bitmap"):
        i, u = ctypes.c_uint64(0), ctypes.c_uint64(0)
        j = _load().orc_jaccard(self._h, other._h, ctypes.byref(i), ctypes.byref(u))
        return j, int(i.value), int(u.value)

    def cosine(self, other: "Bitmap"):
        i = ctypes.c_uint64(0)
        c = _load().orc_cosine(self._h, other._h, ctypes.byref(i))
        return c, int(i.value)

    def contains(self, values) -> np.ndarray:
        v = np.ascontiguousarray(values, dtype=np.uint32)
        out = np.zeros(v.size, dtype=np.uint8)
        if v.size:
            _load().orc_contains(self._h, v.ctypes.data, v.size, out.ctypes.data)
        return out

    @staticmethod
    def multi(op: int, inputs) -> "Bitmap":
        arr = (ctypes.c_void_p * max(1, len(inputs)))(*[b._h for b in inputs])
        h = _load().orc_multi(op, arr, len(inputs))
        if not h:
            raise MemoryError("oracle allocation failed")
        return Bitmap(h)

    @property
    def card(self) -> int:
        return int(_load().orc_card(self._h))

    @property
    def n_containers(self) -> int:
        return int(_load().orc_n(self._h))

    def to_u32(self) -> np.ndarray:
        n = self.card
        out = np.empty(n, dtype=np.uint32)
        if n:
            _load().orc_to_u32(self._h, out.ctypes.data, n)
        return out

    def layout(self) -> dict:
        """keys u16, types u8, cards u32, offs u64[n+1], payload u8."""
        lib = _load()
        n = self.n_containers
        keys = np.empty(n, np.uint16)
        types = np.empty(n, np.uint8)
        cards = np.empty(n, np.uint32)
        offs = np.empty(n + 1, np.uint64)
        payload = np.empty(int(lib.orc_payload_bytes(self._h)), np.uint8)
        lib.orc_export(self._h, keys.ctypes.data, types.ctypes.data, cards.ctypes.data,
                       offs.ctypes.data, payload.ctypes.data)
        return {"keys": keys, "types": types, "cards": cards, "offs": offs, "payload": payload}

    def close(self):
        if self._h:
            _load().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
