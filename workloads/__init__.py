"""Seeded synthetic inputs for the Roaring workloads.

This package only draws sorted, distinct uint32 value arrays (and query
lists); it contains none of the Roaring method.  Both the CPU oracle and the
CUDA library build their bitmaps from exactly these arrays, so the two sides
share inputs and nothing else.

The C generator (gen.c) is compiled on first use (or by ``build()``) into
``libgen.so`` next to this file.

Workload recipes (shapes after the paper's Sec. 5 datasets, Table 2, and its
large ClusterData set, App. B):

* ``plain``   two bitmaps, 200 chunks each with 50% key overlap; chunks are a
              third uniform-sparse (c in 1..4096), a third dense (c in
              4097..60000), a third runs (10..200 runs of length 1..500).
* ``sparse``  200 bitmaps over [0, 2^24), c log-uniform 1e3..1e6, uniform values.
* ``runs``    200 bitmaps over [0, 2^26), runs of geometric length (mean 64)
              separated by geometric gaps (mean 256), c log-uniform 1e4..5e6.
* ``batched`` pool of 4096 bitmaps over [0, 2^32), c log-uniform 10..1e7,
              classes 40% uniform-sparse / 30% dense-clustered / 30% runs.
* ``serving`` index of 10,000 bitmaps, c log-uniform 1e2..1e7, same mixture.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so (gcc, portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_bitmaps", ctypes.c_uint32),
                ("universe_log2", ctypes.c_uint32), ("log10_lo", ctypes.c_double),
                ("log10_hi", ctypes.c_double), ("pm_sparse", ctypes.c_uint32),
                ("pm_dense", ctypes.c_uint32), ("pm_runs", ctypes.c_uint32),
                ("run_k", ctypes.c_uint32), ("gap_k", ctypes.c_uint32),
                ("d_lo", ctypes.c_double), ("d_hi", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        lib.gen_pool_create.restype = vp
        lib.gen_pool_create.argtypes = [ctypes.POINTER(_Params), ctypes.c_int]
        lib.gen_pool_create_some.restype = vp
        lib.gen_pool_create_some.argtypes = [ctypes.POINTER(_Params), vp, u32, ctypes.c_int]
        lib.gen_plain_pair.restype = vp
        lib.gen_plain_pair.argtypes = [u64]
        lib.gen_pool_free.argtypes = [vp]
        lib.gen_pool_n.restype = u32
        lib.gen_pool_n.argtypes = [vp]
        lib.gen_pool_size.restype = u64
        lib.gen_pool_size.argtypes = [vp, u32]
        lib.gen_pool_values.restype = vp
        lib.gen_pool_values.argtypes = [vp, u32]
        lib.gen_pool_class.restype = u32
        lib.gen_pool_class.argtypes = [vp, u32]
        lib.gen_pairs.argtypes = [u64, u64, u32, u32, u32, u32, vp, vp, vp]
        lib.gen_multi_queries.argtypes = [u64, u64, u32, u32, u32, vp, vp, vp, vp]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class PoolSpec:
    """Recipe of a pool of bitmaps (see the module docstring)."""
    seed: int
    n_bitmaps: int
    universe_log2: int
    log10_lo: float
    log10_hi: float
    pm_sparse: int = 1000
    pm_dense: int = 0
    pm_runs: int = 0
    run_k: int = 6          # run length ~ Geom(mean 2^6 = 64)
    gap_k: int = 8          # gap length ~ Geom(mean 2^8 = 256)
    d_lo: float = 0.02
    d_hi: float = 0.9


SPECS = {
    "sparse": PoolSpec(seed=2, n_bitmaps=200, universe_log2=24, log10_lo=3.0, log10_hi=6.0),
    "runs": PoolSpec(seed=3, n_bitmaps=200, universe_log2=26, log10_lo=4.0,
                     log10_hi=6.698970004336019, pm_sparse=0, pm_runs=1000),
    "batched": PoolSpec(seed=4, n_bitmaps=4096, universe_log2=32, log10_lo=1.0, log10_hi=7.0,
                        pm_sparse=400, pm_dense=300, pm_runs=300),
    "serving": PoolSpec(seed=5, n_bitmaps=10000, universe_log2=32, log10_lo=2.0, log10_hi=7.0,
                        pm_sparse=400, pm_dense=300, pm_runs=300),
}

# batched op mix, per mille thresholds: AND 40%, OR 30%, ANDNOT 15%, XOR 15%
BATCHED_OP_MIX = (400, 700, 850)


def scaled(spec: PoolSpec, n_bitmaps: int | None = None, log10_hi: float | None = None,
           seed: int | None = None) -> PoolSpec:
    """A smaller pool with the same shape (fewer bitmaps and/or a lower top cardinality)."""
    kw = {}
    if n_bitmaps is not None:
        kw["n_bitmaps"] = n_bitmaps
    if log10_hi is not None:
        kw["log10_hi"] = log10_hi
    if seed is not None:
        kw["seed"] = seed
    return replace(spec, **kw)


class Pool:
    """A generated pool: ``values(i)`` is a sorted, distinct uint32 numpy view."""

    def __init__(self, handle, lib):
        self._h = handle
        self._lib = lib
        self.n = lib.gen_pool_n(handle)

    def size(self, i: int) -> int:
        return int(self._lib.gen_pool_size(self._h, i))

    def sizes(self) -> np.ndarray:
        return np.array([self.size(i) for i in range(self.n)], dtype=np.uint64)

    def klass(self, i: int) -> int:
        """0 uniform-sparse, 1 dense-clustered, 2 runs."""
        return int(self._lib.gen_pool_class(self._h, i))

    def values(self, i: int) -> np.ndarray:
        n = self.size(i)
        if n == 0:
            return np.zeros(0, dtype=np.uint32)
        ptr = self._lib.gen_pool_values(self._h, i)
        buf = (ctypes.c_uint32 * n).from_address(ptr)
        arr = np.frombuffer(buf, dtype=np.uint32)
        return arr

    def close(self):
        if self._h:
            self._lib.gen_pool_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_pool(spec: PoolSpec, threads: int | None = None) -> Pool:
    lib = _load()
    p = _Params(spec.seed, spec.n_bitmaps, spec.universe_log2, spec.log10_lo, spec.log10_hi,
                spec.pm_sparse, spec.pm_dense, spec.pm_runs, spec.run_k, spec.gap_k,
                spec.d_lo, spec.d_hi)
    h = lib.gen_pool_create(ctypes.byref(p), int(threads or os.cpu_count() or 1))
    if not h:
        raise MemoryError("workload generation failed")
    return Pool(h, lib)


def make_pool_some(spec: PoolSpec, idx, threads: int | None = None) -> Pool:
    """Bitmaps idx of the pool `spec` describes (set j is bitmap idx[j], with
    the same values make_pool(spec) gives it), so that a large pool can be
    drawn a slice at a time."""
    lib = _load()
    p = _Params(spec.seed, spec.n_bitmaps, spec.universe_log2, spec.log10_lo, spec.log10_hi,
                spec.pm_sparse, spec.pm_dense, spec.pm_runs, spec.run_k, spec.gap_k,
                spec.d_lo, spec.d_hi)
    ix = np.ascontiguousarray(idx, dtype=np.uint32)
    h = lib.gen_pool_create_some(ctypes.byref(p), ix.ctypes.data if ix.size else None, ix.size,
                                 int(threads or os.cpu_count() or 1))
    if not h:
        raise MemoryError("workload generation failed (or an index is outside the pool)")
    return Pool(h, lib)


def slices(n: int, step: int):
    """[lo, hi) ranges of step bitmaps covering 0..n."""
    return [(lo, min(n, lo + step)) for lo in range(0, n, step)]


def stream_pool(spec: PoolSpec, consume, step: int = 512, threads: int | None = None):
    """Hand every bitmap of the pool `spec` describes to consume(i, values),
    in index order, drawing step bitmaps at a time and releasing each slice
    before the next (host memory stays at one slice).  Returns (sizes,
    classes) of the whole pool."""
    sizes = np.zeros(spec.n_bitmaps, np.uint64)
    cls = np.zeros(spec.n_bitmaps, np.uint32)
    for lo, hi in slices(spec.n_bitmaps, step):
        part = make_pool_some(spec, np.arange(lo, hi), threads)
        try:
            for j in range(hi - lo):
                sizes[lo + j] = part.size(j)
                cls[lo + j] = part.klass(j)
                consume(lo + j, part.values(j))
        finally:
            part.close()
    return sizes, cls


def plain_pair(seed: int = 1) -> Pool:
    """The two-bitmap workload (seed 1 by default)."""
    lib = _load()
    h = lib.gen_plain_pair(seed)
    if not h:
        raise MemoryError("workload generation failed")
    return Pool(h, lib)


def pairs(seed: int, n_pairs: int, pool_n: int, mix=BATCHED_OP_MIX):
    """(op, a, b) uint32 arrays; op 0 AND, 1 OR, 2 ANDNOT, 3 XOR; a != b."""
    lib = _load()
    op = np.empty(n_pairs, np.uint32)
    a = np.empty(n_pairs, np.uint32)
    b = np.empty(n_pairs, np.uint32)
    lib.gen_pairs(seed, n_pairs, pool_n, mix[0], mix[1], mix[2],
                  op.ctypes.data, a.ctypes.data, b.ctypes.data)
    return op, a, b


def multi_queries(seed: int, nq: int, pool_n: int, k_lo: int = 2, k_hi: int = 8):
    """Multi-way queries: (op 0 AND / 1 OR, k, count_only, members[nq, k_hi])."""
    lib = _load()
    op = np.empty(nq, np.uint32)
    k = np.empty(nq, np.uint32)
    co = np.empty(nq, np.uint32)
    mem = np.empty((nq, k_hi), np.uint32)
    lib.gen_multi_queries(seed, nq, pool_n, k_lo, k_hi, op.ctypes.data, k.ctypes.data,
                          co.ctypes.data, mem.ctypes.data)
    return op, k, co, mem


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream; timing only, never results."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
