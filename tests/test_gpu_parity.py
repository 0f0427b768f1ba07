"""GPU parity: the CUDA path against the CPU oracle, bit for bit, as decoded
uint32 sets and as canonical container layouts (keys, types, cardinalities,
payload bytes).  All of this is integer work: the tolerance is zero."""
import numpy as np
import pytest

from layout_tools import check_canonical

pytestmark = pytest.mark.gpu

OPS = (0, 1, 2, 3)
NP_OPS = {0: np.intersect1d, 1: np.union1d, 2: lambda a, b: np.setdiff1d(a, b, assume_unique=True),
          3: lambda a, b: np.setxor1d(a, b, assume_unique=True)}


@pytest.fixture(scope="module")
def rb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def assert_layout_eq(got, exp, ctx=""):
    for k in ("keys", "types", "cards", "offs", "payload"):
        assert got[k].shape == exp[k].shape, (ctx, k, got[k].shape, exp[k].shape)
        if not np.array_equal(got[k], exp[k]):
            bad = np.nonzero(got[k] != exp[k])[0][:5]
            raise AssertionError(f"{ctx}: {k} differs at {bad}: {got[k][bad]} vs {exp[k][bad]}")


def chunk(rng, key, kind, size):
    """Values of one chunk of a given container kind and size class."""
    base = np.uint32(key) << np.uint32(16)
    if kind == "array":
        c = int(rng.integers(1, 12)) if size == "small" else int(rng.integers(300, 4097))
        v = rng.choice(65536, size=c, replace=False)
    elif kind == "bitset":
        c = int(rng.integers(4097, 40000))
        v = rng.choice(65536, size=c, replace=False)
    else:
        nr = int(rng.integers(1, 10)) if size == "small" else int(rng.integers(40, 600))
        starts = np.sort(rng.choice(65536 // 32, size=nr, replace=False)) * 32
        lens = rng.integers(2, 30, size=nr)
        v = np.unique(np.concatenate([np.arange(s, min(65536, s + l)) for s, l in zip(starts, lens)]))
    return (base | np.sort(v).astype(np.uint32)).astype(np.uint32)


def build_pair(rb, orc, a, b):
    return (rb.Bitmap.from_sorted(a), rb.Bitmap.from_sorted(b), orc.Bitmap.from_sorted(a),
            orc.Bitmap.from_sorted(b))


def test_fig1_on_gpu(rb, orc):
    arr = np.arange(1000, dtype=np.uint32) * 62
    runs = np.concatenate([np.arange(2**16, 2**16 + 100), np.arange(2**16 + 101, 2**16 + 201),
                           np.arange(2**16 + 300, 2**16 + 400)]).astype(np.uint32)
    evens = np.arange(2 * 2**16, 3 * 2**16, 2, dtype=np.uint32)
    v = np.concatenate([arr, runs, evens])
    g = rb.Bitmap.from_sorted(v)
    lay = g.layout()
    assert lay["keys"].tolist() == [0, 1, 2] and lay["types"].tolist() == [0, 2, 1]
    assert lay["cards"].tolist() == [1000, 300, 32768]
    assert_layout_eq(lay, orc.Bitmap.from_sorted(v).layout(), "fig1")
    assert np.array_equal(g.to_numpy(), v)
    assert np.array_equal(g.to_tensor().cpu().numpy().view(np.uint32), v)


@pytest.mark.parametrize("ka", ["array", "bitset", "run"])
@pytest.mark.parametrize("kb", ["array", "bitset", "run"])
@pytest.mark.parametrize("size", ["small", "large"])
def test_container_pair_classes(rb, orc, ka, kb, size):
    """Every type pair x op, on one shared key plus unmatched keys on each side."""
    kinds, sizes = ("array", "bitset", "run"), ("small", "large")
    rng = np.random.default_rng(3000 + 100 * kinds.index(ka) + 10 * kinds.index(kb) + sizes.index(size))
    a = np.concatenate([chunk(rng, 1, ka, size), chunk(rng, 7, ka, size), chunk(rng, 9, "array", "small")])
    b = np.concatenate([chunk(rng, 3, kb, size), chunk(rng, 7, kb, size), chunk(rng, 12, "run", "small")])
    A, B, OA, OB = build_pair(rb, orc, a, b)
    assert_layout_eq(A.layout(), OA.layout(), "build A")
    for op in OPS:
        got = A.op(op, B).layout()
        assert_layout_eq(got, OA.op(op, OB).layout(), f"{ka}x{kb} {size} op{op}")
        check_canonical(got)
        assert A.op_card(op, B) == OA.op_card(op, OB)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_sets(rb, orc, seed):
    from test_oracle import random_set
    r = np.random.default_rng(500 + seed)
    a, b = random_set(r, 5), random_set(r, 5)
    A, B, OA, OB = build_pair(rb, orc, a, b)
    assert_layout_eq(A.layout(), OA.layout(), "build")
    assert np.array_equal(A.to_numpy(), a)
    for op in OPS:
        R = A.op(op, B)
        assert np.array_equal(R.to_numpy(), NP_OPS[op](a, b).astype(np.uint32))
        assert_layout_eq(R.layout(), OA.op(op, OB).layout(), f"op{op}")
    j, i, u = A.jaccard(B)
    assert (j, i, u) == OA.jaccard(OB)


def test_plain_workload(rb, orc, workloads_mod):
    pool = workloads_mod.plain_pair(1)
    a, b = pool.values(0), pool.values(1)
    A, B, OA, OB = build_pair(rb, orc, a, b)
    assert_layout_eq(A.layout(), OA.layout(), "A")
    assert_layout_eq(B.layout(), OB.layout(), "B")
    for op in OPS:
        assert_layout_eq(A.op(op, B).layout(), OA.op(op, OB).layout(), f"op{op}")
        assert A.op_card(op, B) == OA.op_card(op, OB)
    assert A.jaccard(B) == OA.jaccard(OB)


def test_edges(rb, orc):
    e = rb.Bitmap.from_sorted(np.zeros(0, np.uint32))
    assert e.card == 0 and e.n_containers == 0 and e.to_numpy().size == 0
    top_v = np.array([0, 65535, 65536, 0xFFFF0000, 0xFFFFFFFF], np.uint32)
    full = np.arange(5 * 65536, 6 * 65536, dtype=np.uint32)            # <0,65535> run
    t4096 = np.arange(0, 8192, 2, dtype=np.uint32) + 7 * 65536          # 4096 -> array
    t4097 = np.arange(0, 8194, 2, dtype=np.uint32) + 8 * 65536          # 4097 -> bitset
    v = np.concatenate([top_v[:3], full, t4096, t4097, top_v[3:]])
    T = rb.Bitmap.from_sorted(v)
    OT = orc.Bitmap.from_sorted(v)
    assert_layout_eq(T.layout(), OT.layout(), "edges")
    assert T.layout()["types"].tolist() == [0, 0, 2, 0, 1, 0]
    OE = orc.Bitmap.from_sorted(np.zeros(0, np.uint32))
    for op in OPS:
        assert_layout_eq(T.op(op, e).layout(), OT.op(op, OE).layout(), f"x op empty {op}")
        assert_layout_eq(e.op(op, T).layout(), OE.op(op, OT).layout(), f"empty op x {op}")
        assert_layout_eq(T.op(op, T).layout(), OT.op(op, OT).layout(), f"self {op}")
    assert T.op(3, T).n_containers == 0 and T.op(2, T).card == 0
    assert e.jaccard(e) == (0.0, 0, 0)
    with pytest.raises(rb.RoaringError) as ei:
        rb.Bitmap.from_sorted(np.array([5, 3], np.uint32))
    assert ei.value.status == rb.EINVAL
    with pytest.raises(rb.RoaringError):
        rb.Bitmap.from_sorted(np.array([5, 5], np.uint32))


def test_schedules_agree(rb, orc):
    """Lane-sized and warp-sized processing give identical results."""
    from test_oracle import random_set
    r = np.random.default_rng(77)
    a, b = random_set(r, 6), random_set(r, 6)
    A, B, OA, OB = build_pair(rb, orc, a, b)
    saved = rb.get_schedule()
    try:
        for w, c, s in [(2, 6, 0), (4, 3, 32), (8, 1, 2047)]:
            rb.set_schedule(w, c, s)
            for op in OPS:
                assert_layout_eq(A.op(op, B).layout(), OA.op(op, OB).layout(), f"sched {w},{c},{s} op{op}")
    finally:
        rb.set_schedule(saved["warps_per_cta"], saved["ctas_per_sm"], saved["small_intervals"],
                        saved["lean_ctas_per_sm"], saved["prefetch_lines"], saved["tiles_per_take"])


def _pool(workloads_mod, name, n, hi, seed=None):
    spec = workloads_mod.scaled(workloads_mod.SPECS[name], n_bitmaps=n, log10_hi=hi, seed=seed)
    return workloads_mod.make_pool(spec)


@pytest.mark.parametrize("name,n,hi", [("sparse", 24, 5.0), ("runs", 16, 5.3), ("batched", 48, 5.2)])
def test_batch_matches_oracle_and_per_pair(rb, orc, workloads_mod, name, n, hi):
    pool = _pool(workloads_mod, name, n, hi)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    for i in range(0, pool.n, 5):
        assert_layout_eq(G[i].layout(), O[i].layout(), f"build {i}")
    ops, a, b = workloads_mod.pairs(9, 160, pool.n)
    flags = np.zeros(len(ops), np.uint32)
    flags[::4] = rb.Q_COUNT_ONLY
    outs, counts = rb.batch_op(G, ops, a, b, flags)
    for i in range(len(ops)):
        exp = O[a[i]].op(int(ops[i]), O[b[i]])
        assert counts[i] == exp.card, i
        if flags[i]:
            assert outs[i] is None
            continue
        got = outs[i].layout()
        assert_layout_eq(got, exp.layout(), f"{name} pair {i} op {ops[i]}")
        if i % 10 == 0:
            per = G[a[i]].op(int(ops[i]), G[b[i]]).layout()
            assert_layout_eq(per, got, f"per-pair {i}")
    j, ii, uu = rb.batch_jaccard(G, a, b)
    for i in range(0, len(a), 7):
        oj, oi, ou = O[a[i]].jaccard(O[b[i]])
        assert (ii[i], uu[i]) == (oi, ou) and j[i] == oj
    # the same batch with raw handles, released in one call
    raw, c2 = rb.batch_op(G, ops, a, b, flags, raw=True)
    assert np.array_equal(c2, counts)
    for i in range(0, len(ops), 9):
        if flags[i]:
            assert not raw[i]
            continue
        view = rb.Bitmap(raw[i])
        try:
            assert_layout_eq(view.layout(), outs[i].layout(), f"raw {i}")
        finally:
            view._h = None          # the raw array still owns the handle
    rb.free_handles(raw, len(ops))


def test_plan_graph_replay(rb, orc, workloads_mod):
    pool = _pool(workloads_mod, "batched", 32, 5.0, seed=44)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    ops, a, b = workloads_mod.pairs(3, 200, pool.n)
    plan = rb.Plan(G, ops, a, b)
    first, c1 = plan.run()
    second, c2 = plan.run()           # CUDA graph replay
    third, c3 = plan.run()
    assert np.array_equal(c1, c2) and np.array_equal(c1, c3)
    for i in range(0, len(ops), 3):
        exp = O[a[i]].op(int(ops[i]), O[b[i]]).layout()
        assert_layout_eq(first[i].layout(), exp, f"run1 {i}")
        assert_layout_eq(third[i].layout(), exp, f"run3 {i}")
    st = plan.stats()
    assert st["alg_bytes"] > 0 and st["kernel_ms"] > 0


@pytest.mark.parametrize("op", [0, 1])
def test_multi_way(rb, orc, workloads_mod, op):
    pool = _pool(workloads_mod, "sparse", 12, 5.0, seed=12)
    vals = [pool.values(i) for i in range(pool.n)]
    if op == 0:   # make the intersection non-trivial
        common = np.arange(0, 2**24, 97, dtype=np.uint32)
        vals = [np.union1d(v, common).astype(np.uint32) for v in vals]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    for k in (1, 2, 5, 12):
        m, card = rb.multi_op(op, G[:k])
        exp = orc.Bitmap.multi(op, O[:k])
        assert card == exp.card
        assert_layout_eq(m.layout(), exp.layout(), f"multi op{op} k{k}")
        _, c2 = rb.multi_op(op, G[:k], count_only=True)
        assert c2 == exp.card
    m, card = rb.multi_op(op, [])
    assert card == 0


def test_multi_way_mixed_types(rb, orc, workloads_mod):
    pool = _pool(workloads_mod, "batched", 16, 5.5, seed=21)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    # up to 8 members take the per-tile container lookup with lane merges,
    # more members the general path
    for k in (2, 3, 8, 16):
        for op in (0, 1):
            m, card = rb.multi_op(op, G[:k])
            exp = orc.Bitmap.multi(op, O[:k])
            assert card == exp.card
            assert_layout_eq(m.layout(), exp.layout(), f"mixed op{op} k{k}")
            _, c2 = rb.multi_op(op, G[:k], count_only=True)
            assert c2 == exp.card


def test_wide_union_and_intersection_of_200(rb, orc, workloads_mod):
    """Sec. 5 "Wide unions": the union of all 200 bitmaps of the sparse
    workload (cardinalities scaled to at most 10^4.5 so that the oracle's
    sequential fold stays fast), and the intersection of bitmaps that share
    a common subset, each in one multi-way evaluation."""
    pool = _pool(workloads_mod, "sparse", 200, 4.5)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    m, card = rb.multi_op(1, G)
    exp = orc.Bitmap.multi(1, O)
    assert card == exp.card
    assert_layout_eq(m.layout(), exp.layout(), "wide OR of 200")
    common = np.arange(5, 2**24, 61, dtype=np.uint32)
    V2 = [np.union1d(v, common).astype(np.uint32) for v in vals[:40]]
    G2 = [rb.Bitmap.from_sorted(v) for v in V2]
    O2 = [orc.Bitmap.from_sorted(v) for v in V2]
    m2, c2 = rb.multi_op(0, G2)
    exp2 = orc.Bitmap.multi(0, O2)
    assert c2 == exp2.card
    assert_layout_eq(m2.layout(), exp2.layout(), "wide AND of 40")


def test_membership_and_cosine(rb, orc, workloads_mod):
    """Batch membership (host and device values) and the cosine similarity
    against the oracle, on a mixed pool: every container type, values inside
    and just outside each chunk."""
    import torch
    pool = _pool(workloads_mod, "batched", 12, 5.5, seed=33)
    vals = [pool.values(i) for i in range(pool.n)]
    rng = np.random.default_rng(34)
    for i in range(pool.n):
        G, O = rb.Bitmap.from_sorted(vals[i]), orc.Bitmap.from_sorted(vals[i])
        v = vals[i]
        q = np.concatenate([v[::7], (v[::11] + 1).astype(np.uint32), (v[::13] - 1).astype(np.uint32),
                            rng.integers(0, 2**32, 3000, dtype=np.uint64).astype(np.uint32),
                            np.array([0, 65535, 65536, 0xFFFFFFFF], np.uint32)]).astype(np.uint32)
        exp = O.contains(q)
        assert np.array_equal(G.contains(q), exp), i
        dq = torch.from_numpy(q.view(np.int32)).cuda()
        got = G.contains(dq)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), exp), i
        if len(v):
            assert (int(v[len(v) // 2]) in G) and (int(v[0]) in G)
    for i in range(pool.n - 1):
        A, B = rb.Bitmap.from_sorted(vals[i]), rb.Bitmap.from_sorted(vals[i + 1])
        OA, OB = orc.Bitmap.from_sorted(vals[i]), orc.Bitmap.from_sorted(vals[i + 1])
        assert A.cosine(B) == OA.cosine(OB), i
        assert A.cosine(A) == OA.cosine(OA), i
    e = rb.Bitmap.from_sorted(np.zeros(0, np.uint32))
    assert e.contains(np.array([0, 5], np.uint32)).tolist() == [0, 0]
    assert e.cosine(e) == (0.0, 0)


def test_serialize_roundtrip(rb, orc, workloads_mod):
    """The byte image rb_serialize writes equals the one composed from the
    oracle's layout by the documented format; rb_deserialize of it gives the
    same canonical layout, and operations on it match the oracle."""
    from layout_tools import image_from_layout
    pool = _pool(workloads_mod, "batched", 10, 5.5, seed=41)
    vals = [pool.values(i) for i in range(pool.n)] + [np.zeros(0, np.uint32), fig1_like()]
    back = []
    for i, v in enumerate(vals):
        G, O = rb.Bitmap.from_sorted(v), orc.Bitmap.from_sorted(v)
        img = G.serialize()
        assert img == image_from_layout(O.layout()), i
        D = rb.Bitmap.deserialize(img)
        assert_layout_eq(D.layout(), O.layout(), f"roundtrip {i}")
        assert D.card == O.card
        back.append((D, O))
    for i in range(len(back) - 1):
        (D1, O1), (D2, O2) = back[i], back[i + 1]
        for op in OPS:
            assert_layout_eq(D1.op(op, D2).layout(), O1.op(op, O2).layout(), f"op {op} on {i}")


def fig1_like():
    arr = np.arange(1000, dtype=np.uint32) * 62
    runs = np.concatenate([np.arange(2**16, 2**16 + 100), np.arange(2**16 + 101, 2**16 + 201),
                           np.arange(2**16 + 300, 2**16 + 400)]).astype(np.uint32)
    evens = np.arange(2 * 2**16, 3 * 2**16, 2, dtype=np.uint32)
    return np.concatenate([arr, runs, evens])


def test_plan_launch_and_collect(rb, orc, workloads_mod):
    """Two plans launched back to back on one stream and collected later give
    the same results as synchronous runs and as the oracle."""
    pool = _pool(workloads_mod, "batched", 24, 5.2, seed=71)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    ops, a, b = workloads_mod.pairs(7, 120, pool.n)
    pm = rb.Plan(G, ops, a, b)
    pj = rb.Plan(G, np.zeros(len(ops), np.uint32), a, b, np.full(len(ops), rb.Q_COUNT_ONLY, np.uint32))
    ref, cref = pm.run()
    _, jref = pj.run(want_bitmaps=False)
    for rnd in range(3):              # the first launch sizes exactly, later ones replay graphs
        pm.launch()
        pj.launch()
        with pytest.raises(rb.RoaringError):
            pm.launch()                # one outstanding run per plan
        with pytest.raises(rb.RoaringError) as ei:
            pm.run()                   # the launched run owns the plan until collected
        assert ei.value.status == rb.EINVAL
        got, c = pm.collect()
        _, j = pj.collect(want_bitmaps=False)
        assert np.array_equal(c, cref) and np.array_equal(j, jref)
        for i in range(0, len(ops), 7):
            assert_layout_eq(got[i].layout(), ref[i].layout(), f"round {rnd} pair {i}")
            assert_layout_eq(got[i].layout(), O[a[i]].op(int(ops[i]), O[b[i]]).layout(), f"oracle {i}")
            assert int(j[i]) == O[a[i]].op_card(0, O[b[i]])
    with pytest.raises(rb.RoaringError):
        pm.collect()                   # nothing launched


def test_readme_example(rb, orc):
    """The usage example of the README, checked against numpy."""
    va = np.arange(0, 1 << 20, 3, dtype=np.uint32)
    vb = np.arange(0, 1 << 20, 5, dtype=np.uint32)
    a = rb.Bitmap.from_sorted(va)
    b = rb.Bitmap.from_sorted(vb)
    c = a & b
    inter = np.intersect1d(va, vb)
    assert c.card == len(inter) and np.array_equal(c.to_numpy(), inter)
    assert a.op_card(rb.OR, b) == len(np.union1d(va, vb))
    j, i, u = a.jaccard(b)
    assert (i, u) == (len(inter), len(np.union1d(va, vb)))
    assert a.cosine(b) == orc.Bitmap.from_sorted(va).cosine(orc.Bitmap.from_sorted(vb))
    assert (15 in c) and (16 not in c)
    assert np.array_equal((a ^ b).to_numpy(), np.setxor1d(va, vb))
    assert np.array_equal((a - b).to_numpy(), np.setdiff1d(va, vb))
    plan = rb.Plan([a, b], ops=[rb.AND, rb.OR], a=[0, 0], b=[1, 1])
    outs, counts = plan.run()
    assert list(counts) == [len(inter), len(np.union1d(va, vb))]
    union, card = rb.multi_op(rb.OR, [a, b, c])
    assert card == len(np.union1d(va, vb)) and np.array_equal(union.to_numpy(), np.union1d(va, vb))
    acc = rb.Accumulator(rb.OR)
    acc.add(a).add(b)
    assert acc.result()[1] == len(np.union1d(va, vb))
    acc.close()
    img = c.serialize()
    assert rb.Bitmap.deserialize(img).card == c.card


def test_autotune_then_results_match_the_oracle(rb, orc, workloads_mod):
    """rb_autotune searches schedules on a plan, installs the fastest, and
    the plan's results under it equal the oracle's (schedules change speed,
    never results)."""
    pool = _pool(workloads_mod, "batched", 40, 5.3, seed=61)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    O = [orc.Bitmap.from_sorted(v) for v in vals]
    ops, a, b = workloads_mod.pairs(62, 240, pool.n)
    plan = rb.Plan(G, ops, a, b)
    saved = rb.get_schedule()
    try:
        best, ms = plan.autotune(reps=1)
        assert ms > 0 and rb.get_schedule() == best
        assert best["small_intervals"] in (32, 48, 64, 96, 128) and best["lean_ctas_per_sm"] in (6, 7, 8)
        assert best["prefetch_lines"] in (0, 2, 4, 8) and best["tiles_per_take"] in (8, 16, 32, 64)
        outs, counts = plan.run()
        for i in range(len(ops)):
            exp = O[a[i]].op(int(ops[i]), O[b[i]])
            assert int(counts[i]) == exp.card, i
            assert_layout_eq(outs[i].layout(), exp.layout(), f"tuned pair {i}")
    finally:
        rb.set_schedule(saved["warps_per_cta"], saved["ctas_per_sm"], saved["small_intervals"],
                        saved["lean_ctas_per_sm"], saved["prefetch_lines"], saved["tiles_per_take"])
        plan.free()
