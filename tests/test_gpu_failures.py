"""Failure paths on the GPU, made without a GPU fault: an allocator that
refuses (RB_ENOMEM at every allocation point, nothing leaked, the context
still usable) and a bounded barrier wait that runs out (RB_ETIMEOUT, the
context still usable)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1709_07821_gb300 as m
    m.build()
    m.lib()
    return m


class Refusing:
    """Delegates to PyTorch's caching allocator for the first `allow`
    allocations and refuses the rest; tracks what it handed out."""

    def __init__(self, allow):
        import torch
        self.torch = torch
        self.allow = allow
        self.calls = 0
        self.live = {}

    def alloc(self, n, stream):
        self.calls += 1
        if self.calls > self.allow:
            return None
        p = self.torch.cuda.caching_allocator_alloc(n, stream=stream)
        self.live[p] = n
        return p

    def release(self, p, n, stream):
        self.live.pop(p, None)
        self.torch.cuda.caching_allocator_delete(p)


def _sets(seed):
    g = np.random.default_rng(seed)
    a = np.unique(g.integers(0, 1 << 22, 40000, dtype=np.uint64)).astype(np.uint32)
    b = np.unique(g.integers(0, 1 << 22, 60000, dtype=np.uint64)).astype(np.uint32)
    return a, b


def _ops_under(rb, A, B, allow):
    """Every public call that allocates, with the allocator refusing after
    `allow` allocations.  Returns the statuses and whether anything leaked."""
    import torch
    R = Refusing(allow)
    st = []
    with rb.allocator(R.alloc, R.release):
        for f in (lambda: A.op(rb.OR, B), lambda: A.op_card(rb.AND, B), lambda: A.jaccard(B),
                  lambda: rb.multi_op(rb.OR, [A, B, A]), lambda: A.to_numpy(),
                  lambda: rb.batch_op([A, B], np.array([0, 1, 3], np.uint32), np.array([0, 0, 1], np.uint32),
                                      np.array([1, 1, 0], np.uint32))):
            R.calls = 0
            try:
                r = f()
                st.append(rb.OK)
                # release results made under the refusing allocator while it is installed
                rs = r if isinstance(r, tuple) else (r,)
                for x in rs:
                    for y in (x if isinstance(x, list) else [x]):
                        if isinstance(y, rb.Bitmap):
                            y.free()
            except rb.RoaringError as e:
                st.append(e.status)
        torch.cuda.synchronize()
    return st, dict(R.live)


def test_enomem_at_every_allocation_point(rb, oracle_mod):
    a, b = _sets(1)
    A, B = rb.Bitmap.from_sorted(a), rb.Bitmap.from_sorted(b)
    seen_ok = False
    for allow in range(0, 8):
        st, live = _ops_under(rb, A, B, allow)
        assert set(st) <= {rb.OK, rb.ENOMEM}, st
        assert not live, f"allow={allow}: {len(live)} allocation(s) leaked"
        seen_ok |= all(s == rb.OK for s in st)
    assert seen_ok, "no allowance let every call through"
    # the context and the default allocator work afterwards
    want = oracle_mod.Bitmap.from_sorted(a).op(oracle_mod.OR, oracle_mod.Bitmap.from_sorted(b)).to_u32()
    assert np.array_equal((A | B).to_numpy(), want)


def test_construction_refused_returns_enomem(rb):
    a, _ = _sets(2)
    R = Refusing(0)
    with rb.allocator(R.alloc, R.release):
        with pytest.raises(rb.RoaringError) as ei:
            rb.Bitmap.from_sorted(a)
    assert ei.value.status == rb.ENOMEM
    assert not R.live
    assert rb.Bitmap.from_sorted(a).card == len(a)


def test_bounded_wait_times_out_and_context_survives(rb):
    import torch
    assert rb.selftest_wait(1 << 20, complete=True) == rb.OK
    assert rb.selftest_wait(1 << 20, complete=False) == rb.ETIMEOUT
    assert "cycle limit" in rb.lib().rb_last_error().decode()
    assert rb.selftest_wait(1 << 20, complete=True) == rb.OK
    x = torch.arange(10, device="cuda")
    assert int(x.sum()) == 45
    a, b = _sets(3)
    A, B = rb.Bitmap.from_sorted(a), rb.Bitmap.from_sorted(b)
    assert A.op_card(rb.AND, B) == len(np.intersect1d(a, b))


def test_selftest_rejects_bad_limit(rb):
    assert rb.selftest_wait(0, complete=True) == rb.EINVAL
    assert rb.selftest_wait((1 << 31) + 1, complete=True) == rb.EINVAL
