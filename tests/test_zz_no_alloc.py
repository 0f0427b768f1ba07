"""The allocation-free decode, rb_to_u32_noalloc, against rb_to_u32.

Some callers cannot allocate device memory: their memory is wholly reserved
by another allocator, or their path must never allocate or free.
rb_to_u32_noalloc serves them from a fixed device array instead of a fresh
allocation.  This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as m
    m.build()
    L = m.lib()
    L.rb_to_u32_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
    L.rb_to_u32_noalloc.restype = ctypes.c_int
    return m


def sample_sets():
    rng = np.random.default_rng(2024)
    fig1 = np.concatenate([np.arange(1000, dtype=np.uint32) * 62,
                           np.arange(2**16, 2**16 + 100), np.arange(2**16 + 101, 2**16 + 201),
                           np.arange(2**16 + 300, 2**16 + 400),
                           np.arange(2 * 2**16, 3 * 2**16, 2)]).astype(np.uint32)
    parts = []
    for k in range(40):
        base = np.uint32(k * 3) << np.uint32(16)
        kind = k % 3
        if kind == 0:
            v = rng.choice(65536, size=int(rng.integers(1, 4000)), replace=False)
        elif kind == 1:
            v = rng.choice(65536, size=int(rng.integers(5000, 30000)), replace=False)
        else:
            s = int(rng.integers(0, 60000))
            v = np.arange(s, s + int(rng.integers(10, 5000)))
        parts.append(base | np.sort(v).astype(np.uint32))
    mixed = np.concatenate(parts).astype(np.uint32)
    top = np.array([0, 1, 65535, 0xFFFF0000, 0xFFFFFFFF], np.uint32)
    return [fig1, mixed, top]


def decode_noalloc(rb, bm, cap, stream, out=None):
    import torch
    if out is None:
        out = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")   # the caller's buffer
    got = ctypes.c_uint64()
    st = rb.lib().rb_to_u32_noalloc(bm._h, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(got),
                                    ctypes.c_void_p(stream))
    return st, got.value, out


def test_noalloc_decode_matches_rb_to_u32_on_two_calls(rb):
    import torch
    sets = sample_sets()
    bms = [rb.Bitmap.from_sorted(v) for v in sets]
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                       # consecutive calls share the scratch array
        for v, bm in zip(sets, bms):
            buf = torch.full((bm.card,), -1, dtype=torch.int32, device="cuda")    # the caller's buffer
            before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
            st, n, out = decode_noalloc(rb, bm, bm.card, stream, buf)
            after = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
            assert st == rb.OK, rb.lib().rb_last_error()
            assert after == before, "the entry point allocated device memory"
            torch.cuda.synchronize()
            assert n == len(v)
            got = out[:n].cpu().numpy().view(np.uint32)
            ref = bm.to_numpy()                 # the existing entry point
            assert np.array_equal(got, ref), f"call {call}"   # integer work: zero tolerance
            assert np.array_equal(got, v)


def test_noalloc_limits(rb):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    many = (np.arange(20000, dtype=np.uint32) << np.uint32(16)) | np.uint32(7)   # 20000 containers
    bm = rb.Bitmap.from_sorted(many)
    st, n, _ = decode_noalloc(rb, bm, bm.card, stream)
    assert st == rb.ERANGE and n == 20000
    small = rb.Bitmap.from_sorted(np.arange(100, dtype=np.uint32))
    st, n, _ = decode_noalloc(rb, small, 50, stream)
    assert st == rb.ERANGE and n == 100


def test_noalloc_at_the_container_limit(rb):
    """16,384 containers (the documented maximum, every entry of the fixed
    array in use) decode exactly as rb_to_u32 does; 16,385 are refused."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for n_cont, want in ((16384, rb.OK), (16385, rb.ERANGE)):
        v = (np.arange(n_cont, dtype=np.uint32) << np.uint32(16)) | (np.arange(n_cont, dtype=np.uint32) % 65536)
        bm = rb.Bitmap.from_sorted(v)
        assert bm.n_containers == n_cont
        st, n, out = decode_noalloc(rb, bm, bm.card, stream)
        assert st == want and n == n_cont, rb.lib().rb_last_error()
        if want == rb.OK:
            torch.cuda.synchronize()
            got = out[:n].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, bm.to_numpy()) and np.array_equal(got, v)
