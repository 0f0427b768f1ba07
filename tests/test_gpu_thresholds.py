"""Canonical-type boundaries of operation OUTPUTS on the GPU, through every
path that decides a result's type, against the oracle's layout bit for bit.

The cases (tests/threshold_cases.py, pinned on the CPU by
test_threshold_cases.py) make a result land on c = 4096 / 4097,
r = 2047 / 2048 with c > 4096, 2r = c and 2r = c -+ 1 with c <= 4096, the
full chunk <0,65535>, and the chunk-edge values 0 and 65535 (Sec. 1's type
constraints).  Their sizes route them to each container-pair path: one-lane
merges and sweeps, 8-lane group merges, warp merges, the heavy kernel's bit
probes (list emit) and tiles (tile emit); the multi-way kernel's one-lane
k-way merges and its tile folds; and the accumulator's tile emit.  Each path
decides the type on its own, so each is checked on its own:

- pairwise calls (rb_apply), one case per call;
- one batch with every case (materialising and count-only);
- all cases of one op as the keys of ONE pair of bitmaps, so that a warp's
  tile mixes every path;
- 2-way and 3-way multi-way AND / OR;
- the in-place accumulator (OR, AND).

A last test runs a work-stealing plan several times and requires every
result's exported bytes to be identical across runs (placement comes from
atomic allocation; the canonical layout must not)."""
import numpy as np
import pytest

from threshold_cases import canon, cases, runs_of, with_keys

pytestmark = pytest.mark.gpu

FIELDS = ("keys", "types", "cards", "offs", "payload")


def key_of(i):
    return 65535 if i % 5 == 1 else (i * 977) % 65536


CASES = with_keys(cases(), key_of)


def assert_layout_eq(got, exp, ctx=""):
    for k in FIELDS:
        assert got[k].shape == exp[k].shape, (ctx, k, got[k].shape, exp[k].shape)
        if not np.array_equal(got[k], exp[k]):
            bad = np.nonzero(got[k] != exp[k])[0][:5]
            raise AssertionError(f"{ctx}: {k} differs at {bad}: {got[k][bad]} vs {exp[k][bad]}")


@pytest.fixture(scope="module")
def rb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_07821_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def built(rb, oracle_mod):
    """Device and oracle bitmaps of every case, and the oracle's result."""
    out = []
    for name, op, a, b, T in CASES:
        OA, OB = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
        exp = OA.op(op, OB)
        low = T & 0xFFFF
        lay = exp.layout()
        assert np.array_equal(exp.to_u32(), T) and int(lay["types"][0]) == canon(len(low), runs_of(low)), name
        out.append((name, op, rb.Bitmap.from_sorted(a), rb.Bitmap.from_sorted(b), OA, OB, lay))
    return out


def test_pairwise_calls(rb, built):
    for name, op, A, B, OA, OB, exp in built:
        R = A.op(op, B)
        assert_layout_eq(R.layout(), exp, name)
        assert A.op_card(op, B) == int(exp["cards"].sum()), name
        R.free()


def test_one_batch_of_every_case(rb, built):
    pool = []
    for _, _, A, B, *_ in built:
        pool += [A, B]
    n = len(built)
    ops = np.array([c[1] for c in built], np.uint32)
    a = np.arange(0, 2 * n, 2, dtype=np.uint32)
    b = a + 1
    outs, counts = rb.batch_op(pool, ops, a, b)
    for i, (name, op, A, B, OA, OB, exp) in enumerate(built):
        assert_layout_eq(outs[i].layout(), exp, "batch " + name)
        assert int(counts[i]) == int(exp["cards"].sum()), name
    # count-only forms (Sec. 5 identities from |A n B|) and Jaccard
    _, cc = rb.batch_op(pool, ops, a, b, np.full(n, rb.Q_COUNT_ONLY, np.uint32))
    assert np.array_equal(cc, counts)
    j, ii, uu = rb.batch_jaccard(pool, a, b)
    for i, (name, op, A, B, OA, OB, exp) in enumerate(built):
        assert (j[i], int(ii[i]), int(uu[i])) == OA.jaccard(OB), name
    # the plan path (CUDA graph replay) gives the same bytes
    plan = rb.Plan(pool, ops, a, b)
    plan.run(want_bitmaps=False)
    again, c2 = plan.run()
    assert np.array_equal(c2, counts)
    for i, (name, *_ , exp) in enumerate(built):
        assert_layout_eq(again[i].layout(), exp, "plan " + name)
    plan.free()


@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_every_case_of_an_op_in_one_pair(rb, oracle_mod, op):
    """All cases of one op as the keys of one pair of bitmaps (one key per
    case): a tile's 32 slots mix lane, group, warp and heavy paths."""
    sel = [c for c in cases() if c[1] == op]
    keyed = with_keys(sel, lambda i: i * 211 % 65536)     # distinct keys
    va = np.sort(np.concatenate([c[2] for c in keyed])).astype(np.uint32)
    vb = np.sort(np.concatenate([c[3] for c in keyed])).astype(np.uint32)
    OA, OB = oracle_mod.Bitmap.from_sorted(va), oracle_mod.Bitmap.from_sorted(vb)
    exp = OA.op(op, OB)
    assert np.array_equal(exp.to_u32(), np.sort(np.concatenate([c[4] for c in keyed])))
    A, B = rb.Bitmap.from_sorted(va), rb.Bitmap.from_sorted(vb)
    assert_layout_eq(A.op(op, B).layout(), exp.layout(), f"op {op} all cases")
    outs, counts = rb.batch_op([A, B], [op, op], [0, 1], [1, 0])
    assert_layout_eq(outs[0].layout(), exp.layout(), f"op {op} all cases, batch")
    assert_layout_eq(outs[1].layout(), OB.op(op, OA).layout(), f"op {op} all cases, swapped")


def test_multi_way_boundaries(rb, oracle_mod, built):
    """2-way and 3-way AND / OR of the cases (one-lane k-way merges for small
    arrays, tile folds otherwise)."""
    for name, op, A, B, OA, OB, exp in built:
        if op not in (0, 1):
            continue
        m, card = rb.multi_op(op, [A, B])
        assert_layout_eq(m.layout(), exp, "multi2 " + name)
        assert card == int(exp["cards"].sum())
        _, c0 = rb.multi_op(op, [A, B], count_only=True)
        assert c0 == card
        # a third member that leaves the result unchanged: AND, the union of
        # both inputs; OR, every fifth value of the result
        if op == 0:
            vc = np.union1d(OA.to_u32(), OB.to_u32()).astype(np.uint32)
        else:
            vc = OA.op(1, OB).to_u32()[::5].copy()
        C, OC = rb.Bitmap.from_sorted(vc), oracle_mod.Bitmap.from_sorted(vc)
        want = oracle_mod.Bitmap.multi(op, [OA, OC, OB]).layout()
        assert_layout_eq(want, exp, "oracle multi3 " + name)
        m3, c3 = rb.multi_op(op, [A, C, B])
        assert_layout_eq(m3.layout(), exp, "multi3 " + name)
        m.free(), m3.free(), C.free()


def test_accumulator_boundaries(rb, built):
    for name, op, A, B, OA, OB, exp in built:
        if op not in (0, 1):
            continue
        acc = rb.Accumulator(op, max_keys=4)
        try:
            acc.add(A).add(B)
            R, card = acc.result()
            assert card == int(exp["cards"].sum()), name
            assert_layout_eq(R.layout(), exp, "accum " + name)
            R.free()
        finally:
            acc.close()


def test_results_are_identical_across_work_stealing_runs(rb, oracle_mod, workloads_mod):
    """A plan whose pairs have very uneven sizes (so that warps steal tiles in
    a different order every run) run three times, plus a fresh batch: every
    result's exported layout is byte-identical across the runs, and a
    sample equals the oracle."""
    spec = workloads_mod.scaled(workloads_mod.SPECS["batched"], n_bitmaps=160, log10_hi=5.8, seed=91)
    pool = workloads_mod.make_pool(spec)
    vals = [pool.values(i) for i in range(pool.n)]
    G = [rb.Bitmap.from_sorted(v) for v in vals]
    ops, a, b = workloads_mod.pairs(92, 1500, pool.n)
    plan = rb.Plan(G, ops, a, b)
    runs = []
    for _ in range(3):
        outs, counts = plan.run()
        runs.append((counts, [o.layout() for o in outs]))
        for o in outs:
            o.free()
    fresh, fc = rb.batch_op(G, ops, a, b)
    runs.append((fc, [o.layout() for o in fresh]))
    c0, l0 = runs[0]
    for r, (c, lays) in enumerate(runs[1:], 1):
        assert np.array_equal(c, c0), r
        for i in range(len(ops)):
            assert_layout_eq(lays[i], l0[i], f"run {r} pair {i}")
    O = {}
    for i in range(0, len(ops), 25):
        for x in (int(a[i]), int(b[i])):
            if x not in O:
                O[x] = oracle_mod.Bitmap.from_sorted(vals[x])
        assert_layout_eq(l0[i], O[int(a[i])].op(int(ops[i]), O[int(b[i])]).layout(), f"oracle pair {i}")
    plan.free()
