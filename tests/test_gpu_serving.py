"""Serving loop: continuous batching over a device-resident index.  Each
request's result inside a concurrent, mixed stream must be identical to the
same query run alone and to the oracle's sequential fold (integer sets:
tolerance zero)."""
import threading
import time

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
    spec = W.scaled(W.SPECS["serving"], n_bitmaps=48, log10_hi=5.3)
    pool = W.make_pool(spec)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [oracle_mod.Bitmap.from_sorted(v) for v in vals]
    return rb, oracle_mod, W, pool, G, O


def test_results_alone_equal_results_in_the_mix(env):
    rb, orc, W, pool, G, O = env
    ops, ks, co, mem = W.multi_queries(51, 120, pool.n)
    srv = rb.Server(G, mem_budget=8 << 30, max_inflight_batches=4, max_batch=16)
    try:
        tickets = [srv.submit(int(ops[q]), mem[q, :ks[q]].tolist(), bool(co[q])) for q in range(len(ops))]
        lat = []
        for q, t in enumerate(tickets):
            got, card, latency = srv.wait(t, timeout_ms=60000)
            members = mem[q, :ks[q]].tolist()
            alone, card_alone = rb.multi_op(int(ops[q]), [G[m] for m in members], count_only=bool(co[q]))
            exp = orc.Bitmap.multi(int(ops[q]), [O[m] for m in members])
            assert card == card_alone == exp.card, q
            if co[q]:
                assert got is None
            else:
                lay = got.layout()
                ref = alone.layout()
                for k in ("keys", "types", "cards", "offs", "payload"):
                    assert np.array_equal(lay[k], ref[k]), (q, k)
                    assert np.array_equal(lay[k], exp.layout()[k]), (q, k)
                got.free()
                alone.free()
            assert latency > 0
            lat.append(latency)
        st = srv.stats()
        assert st["completed"] == len(ops)
        assert st["batches"] >= 1
    finally:
        srv.close()


def test_requests_arriving_while_batches_run_are_admitted(env):
    rb, orc, W, pool, G, O = env
    ops, ks, co, mem = W.multi_queries(52, 200, pool.n)
    srv = rb.Server(G, mem_budget=8 << 30, max_inflight_batches=3, max_batch=8)
    results = {}
    try:
        def submitter():
            for q in range(len(ops)):
                results[q] = srv.submit(int(ops[q]), mem[q, :ks[q]].tolist(), True)
                if q % 20 == 0:
                    time.sleep(0.001)
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        for q in range(len(ops)):
            _, card, _ = srv.wait(results[q], timeout_ms=60000, want_bitmap=False)
            assert card == orc.Bitmap.multi(int(ops[q]), [O[m] for m in mem[q, :ks[q]]]).card
        st = srv.stats()
        assert st["completed"] == len(ops) and st["batches"] > 1
    finally:
        srv.close()


def test_admission_by_memory(env):
    rb, orc, W, pool, G, O = env
    big = sorted(range(pool.n), key=lambda i: -G[i].card)[:8]
    # a budget below one request's worst case refuses it outright
    srv = rb.Server(G, mem_budget=1 << 16, max_inflight_batches=2, max_batch=4)
    try:
        with pytest.raises(rb.RoaringError) as ei:
            srv.submit(rb.OR, big)
        assert ei.value.status == rb.EBUSY
        t = srv.submit(rb.OR, big, count_only=True)            # count-only needs no result memory
        _, card, _ = srv.wait(t)
        assert card == orc.Bitmap.multi(1, [O[m] for m in big]).card
    finally:
        srv.close()
    # a small budget still serves every request, admitting more as results
    # are freed
    srv = rb.Server(G, mem_budget=256 << 20, max_inflight_batches=2, max_batch=4)
    try:
        ts = [srv.submit(rb.OR, big[i:i + 3]) for i in range(5)]
        for i, t in enumerate(ts):
            bm, card, _ = srv.wait(t, timeout_ms=60000)
            assert card == orc.Bitmap.multi(1, [O[m] for m in big[i:i + 3]]).card
            bm.free()
    finally:
        srv.close()


def test_bad_requests(env):
    rb, orc, W, pool, G, O = env
    srv = rb.Server(G, mem_budget=1 << 30)
    try:
        with pytest.raises(rb.RoaringError):
            srv.submit(rb.XOR, [0, 1])                 # multi-way is AND / OR only
        with pytest.raises(rb.RoaringError):
            srv.submit(rb.AND, [0, pool.n + 5])        # member out of range
        with pytest.raises(rb.RoaringError):
            srv.submit(rb.AND, list(range(9)))         # more than 8 members
    finally:
        srv.close()


def test_bulk_submit_and_poll(env):
    """Requests handed over in bursts (rb_server_submit_many) and collected
    in bursts (rb_server_poll) give the same results as each request alone
    and as the oracle; every ticket comes back exactly once."""
    rb, orc, W, pool, G, O = env
    ops, ks, co, mem = W.multi_queries(53, 150, pool.n)
    srv = rb.Server(G, mem_budget=8 << 30, max_inflight_batches=4, max_batch=32)
    try:
        tickets = np.concatenate([srv.submit_many(ops[i:i + 37], ks[i:i + 37], co[i:i + 37], mem[i:i + 37])
                                  for i in range(0, len(ops), 37)])
        assert len(np.unique(tickets)) == len(ops)
        seen = {}
        while len(seen) < len(ops):
            t, st, cards, lat, bms = srv.poll(cap=16, timeout_ms=60000, want_bitmaps=True)
            assert len(t) > 0
            for x, s, c, l, bm in zip(t, st, cards, lat, bms):
                assert s == 0 and l > 0 and int(x) not in seen
                seen[int(x)] = (int(c), bm)
        for q in range(len(ops)):
            card, bm = seen[int(tickets[q])]
            members = mem[q, :ks[q]].tolist()
            exp = orc.Bitmap.multi(int(ops[q]), [O[m] for m in members])
            assert card == exp.card, q
            if co[q]:
                assert bm is None
            else:
                lay, ref = bm.layout(), exp.layout()
                for k in ("keys", "types", "cards", "offs", "payload"):
                    assert np.array_equal(lay[k], ref[k]), (q, k)
                bm.free()
        t, _, _, _, _ = srv.poll(cap=4, timeout_ms=10)
        assert len(t) == 0
        with pytest.raises(rb.RoaringError):
            srv.submit_many([rb.XOR], [2], [0], np.zeros((1, 8), np.uint32))
    finally:
        srv.close()


def test_results_outlive_the_server(env):
    """Result bitmaps stay valid and freeable after the serving loop (and its
    streams) are gone."""
    rb, orc, W, pool, G, O = env
    ops, ks, co, mem = W.multi_queries(54, 24, pool.n)
    srv = rb.Server(G, mem_budget=8 << 30, max_inflight_batches=3, max_batch=8)
    kept = []
    try:
        tickets = srv.submit_many(ops, ks, np.zeros(len(ops), np.uint32), mem)
        for q, t in enumerate(tickets):
            bm, card, _ = srv.wait(int(t), timeout_ms=60000)
            kept.append((q, bm, card))
    finally:
        srv.close()
    for q, bm, card in kept:
        exp = orc.Bitmap.multi(int(ops[q]), [O[m] for m in mem[q, :ks[q]]])
        assert card == exp.card
        lay, ref = bm.layout(), exp.layout()
        for k in ("keys", "types", "cards", "offs", "payload"):
            assert np.array_equal(lay[k], ref[k]), (q, k)
        bm.free()


def test_wait_beside_concurrent_submits_and_polls(env):
    """rb_server_wait looks its ticket up again after every wake: waiter
    threads block while another thread submits hundreds of requests (the
    ticket map grows through several rehashes), and a ticket that a poll
    collected is reported to a later wait as unknown (RB_EINVAL)."""
    rb, orc, W, pool, G, O = env
    ops, ks, co, mem = W.multi_queries(53, 64, pool.n)
    count = np.ones(len(ops), np.uint8)
    srv = rb.Server(G, mem_budget=8 << 30, max_inflight_batches=4, max_batch=8)
    try:
        tickets = srv.submit_many(ops, ks, count, mem)
        got, errs = {}, []

        def waiter(lo, hi):
            try:
                for q in range(lo, hi):
                    _, card, _ = srv.wait(int(tickets[q]), timeout_ms=120000, want_bitmap=False)
                    got[q] = card
            except Exception as e:   # reported below, on the main thread
                errs.append(e)

        ws = [threading.Thread(target=waiter, args=(16 * i, 16 * (i + 1))) for i in range(4)]
        for w in ws:
            w.start()
        more = sum(len(srv.submit_many(ops, ks, count, mem)) for _ in range(8))
        for w in ws:
            w.join()
        assert not errs, errs
        for q in range(len(ops)):
            assert got[q] == orc.Bitmap.multi(int(ops[q]), [O[m] for m in mem[q, :ks[q]]]).card, q
        seen = 0
        while seen < more:
            t, st, _, _, _ = srv.poll(cap=1024, timeout_ms=120000)
            assert len(t) > 0 and np.all(st == 0)
            seen += len(t)
        t1 = srv.submit(int(ops[0]), mem[0, :ks[0]].tolist(), True)
        collected = []
        while t1 not in collected:
            t, _, _, _, _ = srv.poll(cap=8, timeout_ms=120000)
            assert len(t) > 0
            collected.extend(int(x) for x in t)
        with pytest.raises(rb.RoaringError) as ei:
            srv.wait(t1, timeout_ms=1000)
        assert ei.value.status == rb.EINVAL
    finally:
        srv.close()
