"""Parity at the full size of the batched benchmark workload (4096-bitmap
pool over [0, 2^32), 65,536 pairs), in the launch configuration that
bench.py times: one materialising plan and one count-only plan, each run
once to size its arena and then replayed as a CUDA graph.

- Sampled outputs (seeded, stratified by op and by the input classes) are
  compared with the oracle as canonical layouts, bit for bit.
- Every pair's cardinality is checked against the count-only plan through
  the set identities |A op B| = f(|A|, |B|, |A n B|) (Sec. 5 counts), which
  hold at any size and tie the two independent kernel paths together."""
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


def test_sampled_outputs_match_the_oracle(full, oracle_mod):
    rb, pool, ops, a, b, outs, counts, inter, _ = full
    rng = np.random.default_rng(2024)
    cls = np.array([pool.klass(i) for i in range(pool.n)])
    pick = []
    for op in range(4):                   # every op x (class of a, class of b) stratum, where present
        for ca in range(3):
            for cb in range(3):
                idx = np.nonzero((ops == op) & (cls[a] == ca) & (cls[b] == cb))[0]
                if len(idx):
                    pick.append(int(rng.choice(idx)))
    orc = {}

    def ob(i):
        if i not in orc:
            orc[i] = oracle_mod.Bitmap.from_sorted(pool.values(i))
        return orc[i]

    for i in pick:
        exp = ob(int(a[i])).op(int(ops[i]), ob(int(b[i])))
        assert int(counts[i]) == exp.card, i
        if exp.card == 0:
            assert outs[i].card == 0 and outs[i].n_containers == 0
            continue
        got = outs[i].layout()
        check_canonical(got)
        want = exp.layout()
        for k in ("keys", "types", "cards", "offs", "payload"):
            assert np.array_equal(got[k], want[k]), (i, int(ops[i]), k)


def test_serving_at_full_size(full, oracle_mod, workloads_mod):
    """The serving loop over the full-size pool as its index, in the
    configuration bench.py times (64 GB budget, 4 batches in flight, up to 256
    queries each, bulk submission and polling): every result equals the same
    query run alone, and a stratified sample equals the oracle's fold."""
    rb, pool, ops, a, b, outs, counts, inter, G = full
    mops, ks, co, mem = workloads_mod.multi_queries(5, 300, pool.n)
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
            sample.update(int(i) for i in rng.choice(idx, size=min(3, len(idx)), replace=False))
    orc = {}
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
            for m in mem[q, :ks[q]]:
                if int(m) not in orc:
                    orc[int(m)] = oracle_mod.Bitmap.from_sorted(pool.values(int(m)))
            exp = oracle_mod.Bitmap.multi(int(mops[q]), [orc[int(m)] for m in mem[q, :ks[q]]])
            assert card == exp.card, q
            if not co[q]:
                want = exp.layout()
                for k in ("keys", "types", "cards", "offs", "payload"):
                    assert np.array_equal(bm.layout()[k], want[k]), (q, k)
        if bm is not None:
            bm.free()
        if alone is not None:
            alone.free()
