"""Parity at the full size of the batched benchmark workload (4096-bitmap
pool over [0, 2^32), 65,536 pairs), in the launch configuration that
bench.py times: one materialising plan and one count-only plan, each run
once to size its arena and then replayed as a CUDA graph.

- 2048 sampled outputs (seeded, stratified by op, by the input classes and
  by pair-size decile) are compared with the oracle as canonical layouts,
  bit for bit, and 2048 Jaccard triples from rb_batch_jaccard with the
  oracle's.
- Every pair's cardinality is checked against the count-only plan through
  the set identities |A op B| = f(|A|, |B|, |A n B|) (Sec. 5 counts), which
  hold at any size and tie the two independent kernel paths together.
- The serving loop runs over the serving workload's own index at full size
  (10,000 bitmaps): every result equals the query run alone, and a
  stratified sample equals the oracle's fold."""
import os

import numpy as np
import pytest

from layout_tools import check_canonical

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full(oracle_mod, workloads_mod):
    """The full-size pool on the device with both plans run as bench.py runs them."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as rb
    rb.build()
    pool = workloads_mod.make_pool(workloads_mod.SPECS["batched"])
    ops, a, b = workloads_mod.pairs(4, 65536, pool.n)
    G = [rb.Bitmap.from_sorted(pool.values(i)) for i in range(pool.n)]
    plan_m = rb.Plan(G, ops, a, b)
    plan_j = rb.Plan(G, np.zeros(len(ops), np.uint32), a, b, np.full(len(ops), rb.Q_COUNT_ONLY, np.uint32))
    outs, _ = plan_m.run(raw=True)        # sizes the arena exactly
    plan_m.free_raw(outs)
    plan_j.run(want_bitmaps=False)
    outs, counts = plan_m.run()           # graph replay, as timed by bench.py
    _, inter = plan_j.run(want_bitmaps=False)
    yield rb, pool, ops, a, b, outs, counts, inter, G
    for o in outs:
        if o is not None:
            o.free()
    plan_m.free()
    plan_j.free()


def test_every_cardinality_matches_the_count_identities(full):
    rb, pool, ops, a, b, outs, counts, inter, _ = full
    sz = pool.sizes().astype(np.int64)
    A, B, I = sz[a], sz[b], inter.astype(np.int64)
    want = np.select([ops == 0, ops == 1, ops == 2, ops == 3], [I, A + B - I, A - I, A + B - 2 * I])
    bad = np.nonzero(counts.astype(np.int64) != want)[0]
    assert len(bad) == 0, f"{len(bad)} pairs disagree, first {bad[:5]}"
    # materialising queries always return a handle; an empty result is an
    # empty bitmap
    assert all(o is not None for o in outs)
    for i in np.nonzero(counts == 0)[0][:64]:
        assert outs[i].card == 0 and outs[i].n_containers == 0


N_SAMPLE = 2048


def stratified(rng, ops, a, b, cls, sz, n):
    """n pair indexes spread over every op x class of a x class of b x
    decile of |A| + |B| cell (up to the same number from each cell, the
    rest drawn uniformly)."""
    tot = sz[a] + sz[b]
    dec = np.searchsorted(np.quantile(tot, np.linspace(0, 1, 11)[1:-1]), tot, side="right")
    cell = ((ops * 3 + cls[a]) * 3 + cls[b]) * 10 + dec
    cells = [np.nonzero(cell == c)[0] for c in np.unique(cell)]
    per = max(1, n // len(cells))
    pick = set()
    for idx in cells:
        pick.update(int(i) for i in rng.choice(idx, size=min(per, len(idx)), replace=False))
    rest = np.setdiff1d(np.arange(len(ops)), np.fromiter(pick, np.int64))
    pick.update(int(i) for i in rng.choice(rest, size=max(0, n - len(pick)), replace=False))
    return np.array(sorted(pick))[:n], len(cells)


@pytest.fixture(scope="module")
def oracle_pool(full, oracle_mod):
    """Oracle bitmaps of the whole pool, built on the host cores (ctypes
    releases the GIL, so a thread pool runs them in parallel)."""
    import concurrent.futures as cf
    rb, pool, *_ = full
    with cf.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        O = list(ex.map(lambda i: oracle_mod.Bitmap.from_sorted(pool.values(i)), range(pool.n)))
    yield O
    for o in O:
        o.close()


@pytest.mark.parametrize("n_sample", [N_SAMPLE])
def test_sampled_outputs_match_the_oracle(full, oracle_pool, n_sample):
    """n_sample materialised results of the benchmark's plan, stratified
    over op x input classes x pair-size deciles, equal the oracle's
    canonical layouts byte for byte."""
    import concurrent.futures as cf
    rb, pool, ops, a, b, outs, counts, inter, _ = full
    O = oracle_pool
    cls = np.array([pool.klass(i) for i in range(pool.n)])
    sz = pool.sizes().astype(np.int64)
    pick, n_cells = stratified(np.random.default_rng(2024), ops, a, b, cls, sz, n_sample)
    assert len(pick) == n_sample and n_cells >= 300, (len(pick), n_cells)

    def expect(i):
        r = O[int(a[i])].op(int(ops[i]), O[int(b[i])])
        lay = r.layout()
        r.close()
        return lay

    with cf.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        want = list(ex.map(expect, pick))
    n_nonempty = 0
    for i, w in zip(pick, want):
        assert int(counts[i]) == int(w["cards"].astype(np.int64).sum()), i
        if len(w["keys"]) == 0:
            assert outs[i].card == 0 and outs[i].n_containers == 0, i
            continue
        n_nonempty += 1
        got = outs[i].layout()
        for k in ("keys", "types", "cards", "offs", "payload"):
            assert np.array_equal(got[k], w[k]), (int(i), int(ops[i]), k)
    check_canonical(outs[int(pick[-1])].layout())
    assert n_nonempty > n_sample // 2, n_nonempty


@pytest.mark.parametrize("n_sample", [N_SAMPLE])
def test_sampled_jaccard_matches_the_oracle(full, oracle_pool, n_sample):
    """rb_batch_jaccard over all 65,536 pairs (the public call bench.py
    times end to end); n_sample stratified (|A n B|, |A u B|, J) triples
    equal the oracle's (Sec. 5 "Fast counts"), J as the same correctly
    rounded double, and every |A n B| equals the count-only plan's."""
    import concurrent.futures as cf
    rb, pool, ops, a, b, outs, counts, inter, G = full
    O = oracle_pool
    j, ii, uu = rb.batch_jaccard(G, a, b)
    assert np.array_equal(ii, inter)
    sz = pool.sizes().astype(np.int64)
    assert np.array_equal(uu.astype(np.int64), sz[a] + sz[b] - ii.astype(np.int64))
    cls = np.array([pool.klass(i) for i in range(pool.n)])
    # half stratified as above, half among the pairs that do intersect (most
    # random pairs over [0, 2^32) do not); the expected values are the oracle's
    rng = np.random.default_rng(2025)
    half, _ = stratified(rng, ops, a, b, cls, sz, n_sample // 2)
    meet = np.setdiff1d(np.nonzero(inter > 0)[0], half)
    pick = np.concatenate([half, rng.choice(meet, size=n_sample - len(half), replace=False)])
    with cf.ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        want = list(ex.map(lambda i: O[int(a[i])].jaccard(O[int(b[i])]), pick))
    for i, (wj, wi, wu) in zip(pick, want):
        assert (int(ii[i]), int(uu[i])) == (wi, wu), i
        assert j[i] == wj, i
    assert len(pick) == n_sample and sum(1 for w in want if w[1] > 0) >= n_sample // 2


@pytest.fixture(scope="module")
def serving_index(workloads_mod):
    """The serving workload's index at full size: 10,000 bitmaps drawn and
    uploaded a slice at a time (host memory stays at one slice)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as rb
    rb.build()
    spec = workloads_mod.SPECS["serving"]
    G = []
    sizes, cls = workloads_mod.stream_pool(spec, lambda i, v: G.append(rb.Bitmap.from_sorted(v)))
    yield rb, spec, G, sizes, cls
    for g in G:
        g.free()


def test_serving_index_shape(serving_index):
    """10,000 bitmaps, c log-uniform 1e2..1e7 (log10 mean near 4.5), the
    40/30/30 class mixture, resident on the device."""
    rb, spec, G, sizes, cls = serving_index
    assert len(G) == 10000 and sizes.min() >= 100 and sizes.max() <= 10**7
    assert abs(float(np.log10(sizes.astype(np.float64)).mean()) - 4.5) < 0.1
    frac = np.bincount(cls, minlength=3) / len(cls)
    assert np.all(np.abs(frac - np.array([0.4, 0.3, 0.3])) < 0.03), frac
    for i in range(0, 10000, 997):
        assert G[i].card == int(sizes[i])


def test_serving_at_full_size(serving_index, oracle_mod, workloads_mod):
    """The serving loop over the full 10,000-bitmap index, in the
    configuration bench.py times (64 GB budget, 4 batches in flight, up to
    256 queries each, bulk submission and polling): every result equals the
    same query run alone, and a stratified sample equals the oracle's fold."""
    rb, spec, G, sizes, cls = serving_index
    mops, ks, co, mem = workloads_mod.multi_queries(5, 300, len(G))
    srv = rb.Server(G, mem_budget=64 << 30, max_inflight_batches=4, max_batch=256)
    try:
        tickets = srv.submit_many(mops, ks, co, mem)
        res = {}
        while len(res) < len(mops):
            t, st, cards, _, bms = srv.poll(cap=512, timeout_ms=120000, want_bitmaps=True)
            assert len(t) > 0 and np.all(st == 0)
            for x, c, bm in zip(t, cards, bms):
                res[int(x)] = (int(c), bm)
    finally:
        srv.close()
    rng = np.random.default_rng(7)
    sample = set()
    for op in (0, 1):
        for c in (0, 1):
            idx = np.nonzero((mops == op) & (co == c))[0]
            sample.update(int(i) for i in rng.choice(idx, size=min(4, len(idx)), replace=False))
    need = sorted({int(m) for q in sample for m in mem[q, :ks[q]]})
    host = workloads_mod.make_pool_some(spec, need)
    orc = {m: oracle_mod.Bitmap.from_sorted(host.values(j)) for j, m in enumerate(need)}
    n_checked = 0
    for q in range(len(mops)):
        card, bm = res[int(tickets[q])]
        members = [G[m] for m in mem[q, :ks[q]]]
        alone, card_alone = rb.multi_op(int(mops[q]), members, count_only=bool(co[q]))
        assert card == card_alone, q
        if co[q]:
            assert bm is None
        else:
            got, ref = bm.layout(), alone.layout()
            for k in ("keys", "types", "cards", "offs", "payload"):
                assert np.array_equal(got[k], ref[k]), (q, k)
        if q in sample:
            exp = oracle_mod.Bitmap.multi(int(mops[q]), [orc[int(m)] for m in mem[q, :ks[q]]])
            assert card == exp.card, q
            if not co[q]:
                want = exp.layout()
                for k in ("keys", "types", "cards", "offs", "payload"):
                    assert np.array_equal(bm.layout()[k], want[k]), (q, k)
            n_checked += 1
        if bm is not None:
            bm.free()
        if alone is not None:
            alone.free()
    assert n_checked == len(sample) >= 12
