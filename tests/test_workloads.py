"""The seeded generator: determinism, sortedness and the stated shapes."""
import numpy as np


def test_deterministic_and_sorted(workloads_mod):
    W = workloads_mod
    spec = W.scaled(W.SPECS["batched"], n_bitmaps=24, log10_hi=5.0)
    p1, p2 = W.make_pool(spec, threads=4), W.make_pool(spec, threads=1)
    for i in range(p1.n):
        v1, v2 = p1.values(i), p2.values(i)
        assert np.array_equal(v1, v2)
        assert np.all(np.diff(v1.astype(np.int64)) > 0)
        assert p1.klass(i) == p2.klass(i)
    assert {p1.klass(i) for i in range(p1.n)} <= {0, 1, 2}


def test_plain_pair_shape(workloads_mod):
    pool = workloads_mod.plain_pair(1)
    a, b = pool.values(0), pool.values(1)
    ka, kb = np.unique(a >> 16), np.unique(b >> 16)
    assert len(ka) == 200 and len(kb) == 200
    assert len(np.intersect1d(ka, kb)) == 100
    assert ka.max() < 1024 and kb.max() < 1024


def test_cardinality_law_and_classes(workloads_mod):
    W = workloads_mod
    spec = W.scaled(W.SPECS["sparse"], n_bitmaps=50)
    pool = W.make_pool(spec)
    sizes = pool.sizes()
    assert sizes.min() >= 1000 and sizes.max() <= 1_000_000
    assert all(pool.values(i).max() < 2**24 for i in range(pool.n))
    runs = W.make_pool(W.scaled(W.SPECS["runs"], n_bitmaps=8, log10_hi=5.0))
    for i in range(runs.n):
        v = runs.values(i).astype(np.int64)
        nruns = 1 + np.count_nonzero(np.diff(v) != 1)
        assert len(v) / nruns > 20      # mean run length 64


def test_pairs(workloads_mod):
    op, a, b = workloads_mod.pairs(4, 10000, 4096)
    assert np.all(a != b) and a.max() < 4096 and b.max() < 4096
    frac = np.bincount(op, minlength=4) / len(op)
    assert abs(frac[0] - 0.4) < 0.03 and abs(frac[1] - 0.3) < 0.03
    op2, k, co, mem = workloads_mod.multi_queries(5, 1000, 10000)
    assert k.min() >= 2 and k.max() <= 8
    for q in range(50):
        m = mem[q, :k[q]]
        assert len(np.unique(m)) == k[q]


def test_slices_of_a_pool_equal_the_whole_pool(workloads_mod):
    """make_pool_some draws chosen bitmaps of a pool with the values and
    classes the whole pool gives them (large pools are built a slice at a
    time)."""
    W = workloads_mod
    spec = W.scaled(W.SPECS["serving"], n_bitmaps=40, log10_hi=5.0)
    whole = W.make_pool(spec)
    for lo, hi in W.slices(40, 16):
        part = W.make_pool_some(spec, np.arange(lo, hi))
        for j, i in enumerate(range(lo, hi)):
            assert np.array_equal(part.values(j), whole.values(i)) and part.klass(j) == whole.klass(i)
    pick = W.make_pool_some(spec, [39, 0, 7])
    assert np.array_equal(pick.values(0), whole.values(39))
    import pytest
    with pytest.raises(MemoryError):
        W.make_pool_some(spec, [40])
