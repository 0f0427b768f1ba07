"""In-place accumulation (acc = acc op B over a stream of bitmaps) against
the oracle's sequential fold: the canonical layout of the result after each
add, for OR and AND, over every container type; reset; the tile-pool limit.
Integer sets: the tolerance is zero."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod, workloads_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as rb
    rb.build()
    W = workloads_mod
    pool = W.make_pool(W.scaled(W.SPECS["batched"], n_bitmaps=14, log10_hi=5.5, seed=61))
    vals = [pool.values(i).copy() for i in range(pool.n)]   # copies: the pool is released here
    return rb, oracle_mod, vals


def layouts_equal(got, exp, ctx):
    for k in ("keys", "types", "cards", "offs", "payload"):
        assert np.array_equal(got[k], exp[k]), (ctx, k)


def test_union_in_place(env):
    rb, orc, vals = env
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    acc = rb.Accumulator(rb.OR)
    try:
        for i in range(len(G)):
            acc.add(G[i])
            if i in (0, 1, 4, len(G) - 1):
                exp = orc.Bitmap.multi(1, O[:i + 1])
                bm, card = acc.result()
                assert card == exp.card
                layouts_equal(bm.layout(), exp.layout(), f"OR after {i + 1}")
                assert acc.result(want_bitmap=False)[1] == exp.card
        acc.add(G[3])                                  # adding a member again changes nothing
        layouts_equal(acc.result()[0].layout(), orc.Bitmap.multi(1, O).layout(), "OR again")
        acc.reset()
        assert acc.result()[1] == 0
        acc.add(G[5]).add(G[2])
        layouts_equal(acc.result()[0].layout(), orc.Bitmap.multi(1, [O[5], O[2]]).layout(), "OR after reset")
    finally:
        acc.close()


def test_intersection_in_place(env):
    rb, orc, vals = env
    common = np.unique(np.concatenate([np.arange(0, 2**32 - 1, 9973, dtype=np.uint64),
                                       np.arange(2**20, 2**20 + 70000, dtype=np.uint64)])).astype(np.uint32)
    V = [np.union1d(v, common).astype(np.uint32) for v in vals]
    G = [rb.Bitmap.from_sorted(v) for v in V]
    O = [orc.Bitmap.from_sorted(v) for v in V]
    acc = rb.Accumulator(rb.AND)
    try:
        for i in range(len(G)):
            acc.add(G[i])
            exp = orc.Bitmap.multi(0, O[:i + 1])
            bm, card = acc.result()
            assert card == exp.card
            layouts_equal(bm.layout(), exp.layout(), f"AND after {i + 1}")
        e = rb.Bitmap.from_sorted(np.zeros(0, np.uint32))
        acc.add(e)
        assert acc.result()[1] == 0 and acc.result()[0].n_containers == 0
    finally:
        acc.close()


def test_tile_pool_limit(env):
    rb, orc, vals = env
    big = max(range(len(vals)), key=lambda i: len(np.unique(vals[i] >> 16)))
    n_keys = len(np.unique(vals[big] >> 16))
    acc = rb.Accumulator(rb.OR, max_keys=max(1, n_keys - 1))
    try:
        acc.add(rb.Bitmap.from_sorted(vals[big]))
        with pytest.raises(rb.RoaringError) as ei:
            acc.result()
        assert ei.value.status == rb.ERANGE
    finally:
        acc.close()
    acc = rb.Accumulator(rb.OR, max_keys=n_keys)
    try:
        acc.add(rb.Bitmap.from_sorted(vals[big]))
        layouts_equal(acc.result()[0].layout(), orc.Bitmap.from_sorted(vals[big]).layout(), "exact pool")
    finally:
        acc.close()
