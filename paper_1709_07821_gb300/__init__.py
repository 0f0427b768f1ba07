"""Python binding of librb.so, the GB300 Roaring bitmap library (include/rb.h).

Argument marshalling only: every step of every operation runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory (its caching
allocator is installed as the library's allocator) and the current stream.
If librb.so is missing the first call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librb.so")
_lib = None
_keep = []          # ctypes callbacks that must stay alive

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ERANGE = range(7)
AND, OR, ANDNOT, XOR = 0, 1, 2, 3
ARRAY, BITSET, RUN = 0, 1, 2
Q_COUNT_ONLY = 1
SERVE_MAX_K = 8


class RoaringError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rb status {status}: {msg}")
        self.status = status


class Query(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint32), ("a", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]


class Schedule(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("small_intervals", ctypes.c_uint32), ("lean_ctas_per_sm", ctypes.c_uint32),
                ("prefetch_lines", ctypes.c_uint32), ("tiles_per_take", ctypes.c_uint32)]

    def as_dict(self):
        return {"warps_per_cta": self.warps_per_cta, "ctas_per_sm": self.ctas_per_sm,
                "small_intervals": self.small_intervals, "lean_ctas_per_sm": self.lean_ctas_per_sm,
                "prefetch_lines": self.prefetch_lines, "tiles_per_take": self.tiles_per_take}


class PlanTiming(ctypes.Structure):
    _fields_ = [("lean_ms", ctypes.c_double), ("heavy_ms", ctypes.c_double), ("lean_bytes", ctypes.c_uint64),
                ("heavy_bytes", ctypes.c_uint64), ("alg_bytes", ctypes.c_uint64), ("out_bytes", ctypes.c_uint64),
                ("deferred", ctypes.c_uint64), ("small_ms", ctypes.c_double), ("small_bytes", ctypes.c_uint64),
                ("small_pairs", ctypes.c_uint64)]


class Request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint32), ("k", ctypes.c_uint32), ("count_only", ctypes.c_uint32),
                ("members", ctypes.c_uint32 * SERVE_MAX_K)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)


def build(force: bool = False) -> str:
    """Compile librb.so in-tree for sm_103a (see _build.py)."""
    from . import _build
    return _build.build(force=force)


def _sig(L):
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    pu64, pu32, pdbl = ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_double)
    pvp = ctypes.POINTER(vp)
    spec = {
        "rb_set_allocator": [ALLOC_FN, FREE_FN, vp],
        "rb_from_sorted_u32": [vp, u64, i32, vp, pvp],
        "rb_to_u32": [vp, vp, i32, u64, pu64, vp],
        "rb_cardinality": [vp, pu64],
        "rb_info": [vp, pu32, pu64],
        "rb_export_layout": [vp, vp, vp, vp, vp, vp, u64, vp],
        "rb_apply": [i32, vp, vp, pvp, vp],
        "rb_and": [vp, vp, pvp, vp], "rb_or": [vp, vp, pvp, vp],
        "rb_andnot": [vp, vp, pvp, vp], "rb_xor": [vp, vp, pvp, vp],
        "rb_apply_cardinality": [i32, vp, vp, pu64, vp],
        "rb_and_cardinality": [vp, vp, pu64, vp], "rb_or_cardinality": [vp, vp, pu64, vp],
        "rb_andnot_cardinality": [vp, vp, pu64, vp], "rb_xor_cardinality": [vp, vp, pu64, vp],
        "rb_jaccard": [vp, vp, pdbl, pu64, pu64, vp],
        "rb_cosine": [vp, vp, pdbl, pu64, vp],
        "rb_contains_many": [vp, vp, u64, i32, vp, vp],
        "rb_contains": [vp, u32, ctypes.POINTER(i32)],
        "rb_serialize": [vp, vp, u64, pu64, vp],
        "rb_accum_create": [i32, u32, vp, pvp],
        "rb_accum_add": [vp, vp, vp],
        "rb_accum_result": [vp, pvp, pu64, vp],
        "rb_accum_reset": [vp, vp],
        "rb_deserialize": [vp, u64, vp, pvp],
        "rb_batch_op": [vp, u32, vp, u64, vp, vp, vp],
        "rb_batch_jaccard": [vp, u32, vp, vp, u64, vp, vp, vp, vp],
        "rb_plan_create": [vp, u32, vp, u64, vp, pvp],
        "rb_plan_run": [vp, vp, vp, vp],
        "rb_plan_launch": [vp, vp],
        "rb_plan_collect": [vp, vp, vp],
        "rb_plan_stats": [vp, ctypes.POINTER(PlanTiming)],
        "rb_set_schedule": [ctypes.POINTER(Schedule)],
        "rb_get_schedule": [ctypes.POINTER(Schedule)],
        "rb_autotune": [vp, u32, vp, ctypes.POINTER(Schedule), pdbl],
        "rb_multi_op": [i32, vp, u32, pvp, pu64, vp],
        "rb_server_create": [vp, u32, u64, u32, u32, pvp],
        "rb_server_submit": [vp, ctypes.POINTER(Request), pu64],
        "rb_server_wait": [vp, u64, i32, pvp, pu64, pdbl],
        "rb_server_submit_many": [vp, ctypes.POINTER(Request), u32, pu64],
        "rb_server_poll": [vp, u32, i32, pu64, vp, pvp, pu64, pdbl, pu32],
        "rb_server_stats": [vp, pu64, pu64, pu64],
        "rb_selftest_wait": [u64, ctypes.c_int, vp],
    }
    for name, args in spec.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    for name in ("rb_free", "rb_plan_free", "rb_server_destroy", "rb_accum_free"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = None
    L.rb_free_array.argtypes = [vp, u64]
    L.rb_free_array.restype = None
    L.rb_last_error.restype = ctypes.c_char_p
    L.rb_version.restype = ctypes.c_char_p


def _install_torch_allocator(L):
    import torch

    if not torch.cuda.is_available():
        return

    @ALLOC_FN
    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    @FREE_FN
    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    _keep.extend([_alloc, _free])
    _check(L.rb_set_allocator(_alloc, _free, None))


def lib():
    """The loaded librb.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_1709_07821_gb300.build() "
                               "(nvcc, sm_103a). There is no CPU fallback.")
        L = ctypes.CDLL(LIB_PATH)
        _sig(L)
        _lib = L
        _install_torch_allocator(L)
    return _lib


def _check(st):
    if st != OK:
        raise RoaringError(st, _lib.rb_last_error().decode() if _lib else "")


def _stream(stream=None):
    """A cudaStream_t: stream (a torch.cuda.Stream or a raw handle), else
    PyTorch's current stream."""
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def version() -> str:
    return lib().rb_version().decode()


U32_MAX = 0xFFFFFFFF


def _u32(values, what: str) -> np.ndarray:
    """values as a contiguous uint32 array; raises rather than wrap a value
    outside [0, 2^32) or truncate a non-integer one."""
    v = np.asarray(values)
    if v.size == 0:
        return np.zeros(0, np.uint32)
    if v.dtype.kind not in "iub":
        raise TypeError(f"{what} must be integers, got {v.dtype}")
    if v.dtype.kind == "i" or v.dtype.itemsize > 4:
        lo, hi = int(v.min()), int(v.max())
        if lo < 0 or hi > U32_MAX:
            raise ValueError(f"{what} must lie in [0, 2^32), got values in [{lo}, {hi}]")
    return np.ascontiguousarray(v, dtype=np.uint32)


class Bitmap:
    """Handle on a device-resident canonical Roaring bitmap."""

    __slots__ = ("_h",)

    def __init__(self, handle: int):
        self._h = handle

    # construction -----------------------------------------------------------
    @classmethod
    def from_sorted(cls, values, stream=None) -> "Bitmap":
        """From strictly increasing uint32 values: a numpy array (host) or a
        torch CUDA tensor of 4-byte integers (device)."""
        L = lib()
        h = ctypes.c_void_p()
        if hasattr(values, "is_cuda") and values.is_cuda:
            t = values.contiguous()
            if t.element_size() != 4:
                raise TypeError("device values must be 4-byte integers")
            _check(L.rb_from_sorted_u32(ctypes.c_void_p(t.data_ptr()), t.numel(), 1, _stream(stream),
                                        ctypes.byref(h)))
        else:
            v = _u32(values, "values")
            _check(L.rb_from_sorted_u32(v.ctypes.data if v.size else None, v.size, 0, _stream(stream),
                                        ctypes.byref(h)))
        return cls(h.value)

    # inspection -------------------------------------------------------------
    @property
    def card(self) -> int:
        c = ctypes.c_uint64()
        _check(lib().rb_cardinality(self._h, ctypes.byref(c)))
        return c.value

    def __len__(self):
        return self.card

    @property
    def n_containers(self) -> int:
        n = ctypes.c_uint32()
        _check(lib().rb_info(self._h, ctypes.byref(n), None))
        return n.value

    def payload_bytes(self) -> int:
        p = ctypes.c_uint64()
        _check(lib().rb_info(self._h, None, ctypes.byref(p)))
        return p.value

    def to_numpy(self, stream=None) -> np.ndarray:
        n = self.card
        out = np.empty(n, np.uint32)
        got = ctypes.c_uint64()
        _check(lib().rb_to_u32(self._h, out.ctypes.data if n else None, 0, n, ctypes.byref(got), _stream(stream)))
        return out

    def to_tensor(self, stream=None):
        import torch
        n = self.card
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        got = ctypes.c_uint64()
        _check(lib().rb_to_u32(self._h, ctypes.c_void_p(out.data_ptr()) if n else None, 1, n, ctypes.byref(got),
                               _stream(stream)))
        return out

    def layout(self, stream=None) -> dict:
        """keys u16, types u8, cards u32, offs u64[n+1], payload u8 (canonical)."""
        L = lib()
        n = ctypes.c_uint32()
        p = ctypes.c_uint64()
        _check(L.rb_info(self._h, ctypes.byref(n), ctypes.byref(p)))
        n, p = n.value, p.value
        keys = np.empty(n, np.uint16)
        types = np.empty(n, np.uint8)
        cards = np.empty(n, np.uint32)
        offs = np.empty(n + 1, np.uint64)
        payload = np.empty(p, np.uint8)
        _check(L.rb_export_layout(self._h, keys.ctypes.data, types.ctypes.data, cards.ctypes.data, offs.ctypes.data,
                                  payload.ctypes.data if p else None, p, _stream(stream)))
        return {"keys": keys, "types": types, "cards": cards, "offs": offs, "payload": payload}

    # operations -------------------------------------------------------------
    def op(self, op: int, other: "Bitmap", stream=None) -> "Bitmap":
        h = ctypes.c_void_p()
        _check(lib().rb_apply(op, self._h, other._h, ctypes.byref(h), _stream(stream)))
        return Bitmap(h.value)

    def op_card(self, op: int, other: "Bitmap", stream=None) -> int:
        c = ctypes.c_uint64()
        _check(lib().rb_apply_cardinality(op, self._h, other._h, ctypes.byref(c), _stream(stream)))
        return c.value

    def jaccard(self, other: "Bitmap", stream=None):
        j, i, u = ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().rb_jaccard(self._h, other._h, ctypes.byref(j), ctypes.byref(i), ctypes.byref(u),
                                _stream(stream)))
        return j.value, i.value, u.value

    def cosine(self, other: "Bitmap", stream=None):
        """(|A n B| / sqrt(|A| |B|), |A n B|)."""
        c, i = ctypes.c_double(), ctypes.c_uint64()
        _check(lib().rb_cosine(self._h, other._h, ctypes.byref(c), ctypes.byref(i), _stream(stream)))
        return c.value, i.value

    def contains(self, values, stream=None):
        """Membership of each value: a uint8 array (1 = present).  A CUDA
        torch tensor of uint32/int32 values is answered on the device (the
        result is a CUDA uint8 tensor on the same stream); anything else is
        treated as host values."""
        try:
            import torch
            is_dev = isinstance(values, torch.Tensor) and values.is_cuda
        except Exception:
            is_dev = False
        if is_dev:
            v = values.contiguous()
            if v.dtype not in (torch.int32, torch.uint32):
                raise TypeError("device values must be int32 or uint32")
            out = torch.empty(v.numel(), dtype=torch.uint8, device=v.device)
            _check(lib().rb_contains_many(self._h, v.data_ptr(), v.numel(), 1, out.data_ptr(), _stream(stream)))
            return out
        v = np.asarray(values)
        if v.size and v.dtype.kind not in "iub":
            raise TypeError(f"values must be integers, got {v.dtype}")
        v = v.reshape(-1)
        # a value outside [0, 2^32) is not a member
        if v.dtype.kind == "i" or v.dtype.itemsize > 4:
            inside = (v >= 0) & (v <= U32_MAX)
        else:
            inside = np.ones(v.size, bool)
        out = np.zeros(v.size, dtype=np.uint8)
        w = np.ascontiguousarray(v[inside], dtype=np.uint32)
        if w.size:
            got = np.empty(w.size, dtype=np.uint8)
            _check(lib().rb_contains_many(self._h, w.ctypes.data, w.size, 0, got.ctypes.data, _stream(stream)))
            out[inside] = got
        return out

    def serialize(self, stream=None) -> bytes:
        """The bitmap's portable byte image (format in include/rb.h)."""
        n = ctypes.c_uint64()
        _check(lib().rb_serialize(self._h, None, 0, ctypes.byref(n), _stream(stream)))
        buf = (ctypes.c_uint8 * max(1, n.value))()
        _check(lib().rb_serialize(self._h, buf, n.value, ctypes.byref(n), _stream(stream)))
        return bytes(buf)[:n.value]

    @classmethod
    def deserialize(cls, data: bytes, stream=None) -> "Bitmap":
        buf = (ctypes.c_uint8 * max(1, len(data))).from_buffer_copy(data if data else b"\0")
        h = ctypes.c_void_p()
        _check(lib().rb_deserialize(buf, len(data), _stream(stream), ctypes.byref(h)))
        return cls(h.value)

    def __contains__(self, value):
        value = int(value)
        if not 0 <= value <= U32_MAX:
            return False
        r = ctypes.c_int()
        _check(lib().rb_contains(self._h, int(value), ctypes.byref(r)))
        return bool(r.value)

    def __and__(self, o):
        return self.op(AND, o)

    def __or__(self, o):
        return self.op(OR, o)

    def __sub__(self, o):
        return self.op(ANDNOT, o)

    def __xor__(self, o):
        return self.op(XOR, o)

    # lifetime ---------------------------------------------------------------
    def free(self):
        if self._h:
            if _lib is not None:
                _lib.rb_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _handles(bitmaps):
    return (ctypes.c_void_p * max(1, len(bitmaps)))(*[b._h for b in bitmaps])


def _queries(ops, a, b, flags=None):
    n = len(ops)
    q = (Query * max(1, n))()
    arr = np.frombuffer(q, dtype=np.uint32, count=4 * n).reshape(n, 4) if n else None
    if n:
        arr[:, 0] = _u32(ops, "ops")
        arr[:, 1] = _u32(a, "pool indexes")
        arr[:, 2] = _u32(b, "pool indexes")
        arr[:, 3] = 0 if flags is None else _u32(flags, "flags")
    return q


def batch_op(pool, ops, a, b, flags=None, stream=None, raw=False):
    """Run len(ops) pairwise queries over `pool` in one launch.  Returns
    (bitmaps, counts): bitmaps[i] is None for count-only queries.  With
    raw=True the results stay a ctypes array of library handles (no Python
    object per result); release them with free_handles."""
    n = len(ops)
    q = _queries(ops, a, b, flags)
    outs = (ctypes.c_void_p * max(1, n))()
    counts = np.zeros(n, np.uint64)
    _check(lib().rb_batch_op(_handles(pool), len(pool), q, n, outs, counts.ctypes.data if n else None,
                             _stream(stream)))
    if raw:
        return outs, counts
    return [Bitmap(outs[i]) if outs[i] else None for i in range(n)], counts


def free_handles(outs, n: int):
    """Release n raw result handles (from batch_op(raw=True)) in one call."""
    lib().rb_free_array(outs, n)


def batch_jaccard(pool, a, b, stream=None):
    a = _u32(a, "pool indexes")
    b = _u32(b, "pool indexes")
    if len(a) != len(b):
        raise ValueError("a and b must have the same length")
    n = len(a)
    j = np.zeros(n, np.float64)
    i = np.zeros(n, np.uint64)
    u = np.zeros(n, np.uint64)
    _check(lib().rb_batch_jaccard(_handles(pool), len(pool), a.ctypes.data, b.ctypes.data, n, j.ctypes.data,
                                  i.ctypes.data, u.ctypes.data, _stream(stream)))
    return j, i, u


class Plan:
    """A reusable batch: prepared once, replayed as a CUDA graph per run."""

    def __init__(self, pool, ops, a, b, flags=None, stream=None):
        self._pool = list(pool)
        self.n = len(ops)
        self._q = _queries(ops, a, b, flags)
        h = ctypes.c_void_p()
        _check(lib().rb_plan_create(_handles(self._pool), len(self._pool), self._q, self.n, _stream(stream),
                                    ctypes.byref(h)))
        self._h = h.value

    def run(self, stream=None, want_bitmaps=True, raw=False):
        """Run the batch.  Returns (bitmaps, counts); with raw=True the results
        stay a ctypes array of handles (release it with free_raw), and with
        want_bitmaps=False they are released at once."""
        outs = (ctypes.c_void_p * max(1, self.n))()
        counts = np.zeros(self.n, np.uint64)
        _check(lib().rb_plan_run(self._h, outs, counts.ctypes.data if self.n else None, _stream(stream)))
        if raw:
            return outs, counts
        if not want_bitmaps:
            lib().rb_free_array(outs, self.n)
            return None, counts
        return [Bitmap(outs[i]) if outs[i] else None for i in range(self.n)], counts

    def launch(self, stream=None):
        """Enqueue a run and return at once (collect() finishes it)."""
        _check(lib().rb_plan_launch(self._h, _stream(stream)))

    def collect(self, want_bitmaps=True, raw=False):
        """Wait for the launched run; results as run() returns them."""
        outs = (ctypes.c_void_p * max(1, self.n))()
        counts = np.zeros(self.n, np.uint64)
        _check(lib().rb_plan_collect(self._h, outs, counts.ctypes.data if self.n else None))
        if raw:
            return outs, counts
        if not want_bitmaps:
            lib().rb_free_array(outs, self.n)
            return None, counts
        return [Bitmap(outs[i]) if outs[i] else None for i in range(self.n)], counts

    def free_raw(self, outs):
        """Release the handles of a raw run."""
        lib().rb_free_array(outs, self.n)

    def stats(self):
        t = PlanTiming()
        _check(lib().rb_plan_stats(self._h, ctypes.byref(t)))
        return {"lean_ms": t.lean_ms, "small_ms": t.small_ms, "heavy_ms": t.heavy_ms,
                "kernel_ms": t.lean_ms + t.small_ms + t.heavy_ms, "lean_bytes": t.lean_bytes,
                "small_bytes": t.small_bytes, "heavy_bytes": t.heavy_bytes, "alg_bytes": t.alg_bytes,
                "out_bytes": t.out_bytes, "deferred": t.deferred, "small_pairs": t.small_pairs}

    def autotune(self, reps=2, stream=None):
        s = Schedule()
        ms = ctypes.c_double()
        _check(lib().rb_autotune(self._h, reps, _stream(stream), ctypes.byref(s), ctypes.byref(ms)))
        return s.as_dict(), ms.value

    def free(self):
        if getattr(self, "_h", None):
            lib().rb_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def get_schedule() -> dict:
    s = Schedule()
    _check(lib().rb_get_schedule(ctypes.byref(s)))
    return s.as_dict()


def set_schedule(warps_per_cta: int, ctas_per_sm: int, small_intervals: int, lean_ctas_per_sm: int = 0,
                 prefetch_lines: int = 0, tiles_per_take: int = 32):
    s = Schedule(warps_per_cta, ctas_per_sm, small_intervals, lean_ctas_per_sm, prefetch_lines, tiles_per_take)
    _check(lib().rb_set_schedule(ctypes.byref(s)))


def selftest_wait(limit_cycles: int, complete: bool, stream=None) -> int:
    """Run the bounded-wait self-test; returns the rb_status code (OK or
    ETIMEOUT) rather than raising."""
    return lib().rb_selftest_wait(int(limit_cycles), 1 if complete else 0, _stream(stream))


class allocator:
    """Context manager that routes the library's device allocations through
    alloc(nbytes, stream) -> int pointer or None and release(ptr, nbytes,
    stream), then restores PyTorch's caching allocator."""

    def __init__(self, alloc, release):
        L = lib()

        @ALLOC_FN
        def _a(nbytes, stream, ctx):
            try:
                return alloc(int(nbytes), int(stream or 0))
            except Exception:
                return None

        @FREE_FN
        def _f(ptr, nbytes, stream, ctx):
            try:
                release(int(ptr), int(nbytes), int(stream or 0))
            except Exception:
                pass

        self._fns = (_a, _f)
        self._L = L

    def __enter__(self):
        _keep.extend(self._fns)
        _check(self._L.rb_set_allocator(self._fns[0], self._fns[1], None))
        return self

    def __exit__(self, *exc):
        _install_torch_allocator(self._L)
        return False


def multi_op(op: int, inputs, count_only: bool = False, stream=None):
    """k-way AND / OR.  Returns (bitmap or None, cardinality)."""
    h = ctypes.c_void_p()
    c = ctypes.c_uint64()
    _check(lib().rb_multi_op(op, _handles(inputs), len(inputs), None if count_only else ctypes.byref(h),
                             ctypes.byref(c), _stream(stream)))
    return (None if count_only else Bitmap(h.value)), c.value


class Accumulator:
    """In-place accumulation acc = acc op b (op AND or OR) over many bitmaps,
    with device memory reserved once (max_keys tiles of 8 KB)."""

    def __init__(self, op: int, max_keys: int = 65536, stream=None):
        h = ctypes.c_void_p()
        _check(lib().rb_accum_create(op, max_keys, _stream(stream), ctypes.byref(h)))
        self._h = h.value

    def add(self, b: "Bitmap", stream=None):
        _check(lib().rb_accum_add(self._h, b._h, _stream(stream)))
        return self

    def result(self, want_bitmap: bool = True, stream=None):
        """(bitmap or None, cardinality) of the current state."""
        h = ctypes.c_void_p()
        c = ctypes.c_uint64()
        _check(lib().rb_accum_result(self._h, ctypes.byref(h) if want_bitmap else None, ctypes.byref(c),
                                     _stream(stream)))
        return (Bitmap(h.value) if h.value else None), c.value

    def reset(self, stream=None):
        _check(lib().rb_accum_reset(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().rb_accum_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop over a device-resident index."""

    def __init__(self, index, mem_budget: int, max_inflight_batches: int = 4, max_batch: int = 256):
        self._index = list(index)
        h = ctypes.c_void_p()
        _check(lib().rb_server_create(_handles(self._index), len(self._index), mem_budget, max_inflight_batches,
                                      max_batch, ctypes.byref(h)))
        self._h = h.value

    def submit(self, op: int, members, count_only: bool = False) -> int:
        r = Request()
        r.op = op
        r.k = len(members)          # more than SERVE_MAX_K is refused by the library
        r.count_only = 1 if count_only else 0
        for i, m in enumerate(members[:SERVE_MAX_K]):
            r.members[i] = int(m)
        t = ctypes.c_uint64()
        _check(lib().rb_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    @staticmethod
    def requests(ops, ks, count_only, members) -> np.ndarray:
        """n requests marshalled as rb_request records (one row of
        3 + SERVE_MAX_K uint32 each: op, k, count_only, members), for
        submit_many and submit_prepared."""
        n = len(ops)
        mem = np.asarray(members, dtype=np.int64).reshape(n, -1) if n else np.zeros((0, SERVE_MAX_K), np.int64)
        arr = np.zeros((max(1, n), 3 + SERVE_MAX_K), np.uint32)
        if n:
            arr[:n, 0] = _u32(ops, "ops")
            arr[:n, 1] = _u32(ks, "k")
            arr[:n, 2] = (np.asarray(count_only) != 0).astype(np.uint32)
            w = min(SERVE_MAX_K, mem.shape[1])
            # members past k are not read by the library; keep them in range
            arr[:n, 3:3 + w] = np.where(mem[:, :w] < 0, 0, mem[:, :w] & 0xFFFFFFFF).astype(np.uint32)
        assert ctypes.sizeof(Request) == arr.shape[1] * 4
        return arr

    def submit_prepared(self, reqs: np.ndarray, lo: int, hi: int, tickets: np.ndarray):
        """Queue rows lo..hi of a marshalled request array (Server.requests)
        in one call; tickets[lo:hi] (a uint64 array) receive their tickets."""
        if hi <= lo:
            return
        if not (reqs.flags.c_contiguous and reqs.dtype == np.uint32 and tickets.dtype == np.uint64
                and hi <= len(reqs) and hi <= len(tickets) and lo >= 0):
            raise ValueError("submit_prepared: bad request or ticket array")
        row = reqs.shape[1] * 4
        _check(lib().rb_server_submit_many(self._h, ctypes.cast(ctypes.c_void_p(reqs.ctypes.data + lo * row),
                                                                ctypes.POINTER(Request)), hi - lo,
                                           ctypes.cast(ctypes.c_void_p(tickets.ctypes.data + 8 * lo),
                                                       ctypes.POINTER(ctypes.c_uint64))))

    def submit_many(self, ops, ks, count_only, members) -> np.ndarray:
        """Queue n requests in one call: ops[i], ks[i] members from row i of
        members (an n x SERVE_MAX_K array), count_only[i]; returns the
        tickets (uint64)."""
        n = len(ops)
        t = np.zeros(max(1, n), np.uint64)
        if n:
            self.submit_prepared(self.requests(ops, ks, count_only, members), 0, n, t)
        return t[:n]

    def poll(self, cap: int = 1024, timeout_ms: int = 100, want_bitmaps: bool = False):
        """Up to cap completed requests: (tickets, statuses, cards, latencies
        in seconds, bitmaps or None).  Without want_bitmaps the results are
        freed inside the library."""
        t = np.zeros(cap, np.uint64)
        st = np.zeros(cap, np.int32)
        c = np.zeros(cap, np.uint64)
        lat = np.zeros(cap, np.float64)
        outs = (ctypes.c_void_p * cap)() if want_bitmaps else None
        n = ctypes.c_uint32()
        u64p, dp = ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)
        _check(lib().rb_server_poll(self._h, cap, timeout_ms, t.ctypes.data_as(u64p), st.ctypes.data,
                                    outs, c.ctypes.data_as(u64p), lat.ctypes.data_as(dp), ctypes.byref(n)))
        k = n.value
        bms = [Bitmap(outs[i]) if outs[i] else None for i in range(k)] if want_bitmaps else None
        return t[:k], st[:k], c[:k], lat[:k], bms

    def wait(self, ticket: int, timeout_ms: int = 60000, want_bitmap: bool = True):
        h = ctypes.c_void_p()
        c = ctypes.c_uint64()
        lat = ctypes.c_double()
        _check(lib().rb_server_wait(self._h, ticket, timeout_ms, ctypes.byref(h) if want_bitmap else None,
                                    ctypes.byref(c), ctypes.byref(lat)))
        return (Bitmap(h.value) if h.value else None), c.value, lat.value

    def stats(self):
        c, b, p = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().rb_server_stats(self._h, ctypes.byref(c), ctypes.byref(b), ctypes.byref(p)))
        return {"completed": c.value, "batches": b.value, "peak_inflight": p.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().rb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
