"""Parity at the full sizes of the sparse and run-heavy workloads (200
bitmaps each; the 199 consecutive pairs; the wide union of all 200), in one
batch per operation as the library runs them.

- Every pair's cardinality is tied to the count-only batch by the Sec. 5
  identities, and a seeded sample of pairs is compared with the oracle as
  canonical layouts, bit for bit.
- The wide union of the 200 sparse bitmaps is compared with the canonical
  encoding of the plain union of their values (numpy), which the oracle
  builds directly: the definition, not a fold."""
import numpy as np
import pytest

from layout_tools import check_canonical

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as m
    m.build()
    return m


def layouts_equal(got, want, ctx):
    for k in ("keys", "types", "cards", "offs", "payload"):
        assert np.array_equal(got[k], want[k]), (ctx, k)


def consecutive_pairs(rb, orc, pool, ops_cycle, n_sample, seed):
    n = pool.n
    G = [rb.Bitmap.from_sorted(pool.values(i)) for i in range(n)]
    a = np.arange(n - 1, dtype=np.uint32)
    b = a + 1
    sz = pool.sizes().astype(np.int64)
    _, inter = rb.batch_op(G, np.zeros(n - 1, np.uint32), a, b, np.full(n - 1, rb.Q_COUNT_ONLY, np.uint32))
    I = inter.astype(np.int64)
    rng = np.random.default_rng(seed)
    orc_bm = {}

    def ob(i):
        if i not in orc_bm:
            orc_bm[i] = orc.Bitmap.from_sorted(pool.values(i))
        return orc_bm[i]

    for op in ops_cycle:
        outs, counts = rb.batch_op(G, np.full(n - 1, op, np.uint32), a, b)
        A, B = sz[:-1], sz[1:]
        want = [I, A + B - I, A - I, A + B - 2 * I][op]
        assert np.array_equal(counts.astype(np.int64), want), f"op {op}: count identities"
        for i in rng.choice(n - 1, size=n_sample, replace=False):
            i = int(i)
            exp = ob(i).op(op, ob(i + 1))
            assert int(counts[i]) == exp.card
            got = outs[i].layout()
            check_canonical(got)
            layouts_equal(got, exp.layout(), f"op {op} pair {i}")
        for o in outs:
            o.free()
    return G, I


def test_sparse_full_size(rb, oracle_mod, workloads_mod):
    pool = workloads_mod.make_pool(workloads_mod.SPECS["sparse"])
    G, _ = consecutive_pairs(rb, oracle_mod, pool, (0, 1), 6, 202)
    m, card = rb.multi_op(1, G)
    union = np.unique(np.concatenate([pool.values(i) for i in range(pool.n)])).astype(np.uint32)
    assert card == len(union)
    layouts_equal(m.layout(), oracle_mod.Bitmap.from_sorted(union).layout(), "wide OR of 200")


def test_runs_full_size(rb, oracle_mod, workloads_mod):
    pool = workloads_mod.make_pool(workloads_mod.SPECS["runs"])
    G, I = consecutive_pairs(rb, oracle_mod, pool, (0, 1, 2, 3), 4, 303)
    n = pool.n
    a = np.arange(n - 1, dtype=np.uint32)
    j, inter, uni = rb.batch_jaccard(G, a, a + 1)
    assert np.array_equal(inter.astype(np.int64), I)
    sz = pool.sizes().astype(np.int64)
    assert np.array_equal(uni.astype(np.int64), sz[:-1] + sz[1:] - I)
    for i in (0, n // 2, n - 2):
        oj, oi, ou = oracle_mod.Bitmap.from_sorted(pool.values(i)).jaccard(
            oracle_mod.Bitmap.from_sorted(pool.values(i + 1)))
        assert (int(inter[i]), int(uni[i])) == (oi, ou) and j[i] == oj
