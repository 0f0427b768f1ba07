"""Pins for the CPU oracle: the paper's worked examples, its type thresholds,
its count identities, and brute force on small inputs (numpy's sorted-set
routines).  No GPU needed."""
import json
import os

import numpy as np
import pytest

from layout_tools import check_canonical, decode_layout

GOLD = os.path.join(os.path.dirname(__file__), "golden")
OPS = {0: np.intersect1d, 1: np.union1d, 2: np.setdiff1d, 3: np.setxor1d}


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def ref_op(op, a, b):
    if op in (2, 3):
        return OPS[op](a, b, assume_unique=True).astype(np.uint32)
    return OPS[op](a, b).astype(np.uint32)


def fig1_values():
    arr = np.arange(1000, dtype=np.uint32) * 62
    runs = np.concatenate([np.arange(2**16, 2**16 + 100), np.arange(2**16 + 101, 2**16 + 201),
                           np.arange(2**16 + 300, 2**16 + 400)]).astype(np.uint32)
    evens = np.arange(2 * 2**16, 3 * 2**16, 2, dtype=np.uint32)
    return np.concatenate([arr, runs, evens])


def test_fig1_layout(oracle_mod):
    g = gold("fig1_layout.json")
    bm = oracle_mod.Bitmap.from_sorted(fig1_values())
    lay = bm.layout()
    names = {0: "array", 1: "bitset", 2: "run"}
    assert lay["keys"].tolist() == g["keys"]
    assert [names[t] for t in lay["types"].tolist()] == g["types"]
    assert lay["cards"].tolist() == g["cards"]
    o = lay["offs"]
    arr = lay["payload"][o[0]:o[1]].view(np.uint16)
    assert int(o[1] - o[0]) == g["array_bytes"]
    assert arr[:6].tolist() == g["array_head"] and int(arr[-1]) == g["array_last"]
    runs = lay["payload"][o[1]:o[2]].view(np.uint16).reshape(-1, 2).tolist()
    assert runs == g["runs"]
    words = lay["payload"][o[2]:o[3]].view(np.uint64)
    bits = np.unpackbits(words[:1].view(np.uint8), bitorder="little")[:6].tolist()
    assert bits == g["bitset_first_bits"]
    assert np.all(words == np.uint64(0x5555555555555555))
    check_canonical(lay)
    assert np.array_equal(bm.to_u32(), fig1_values())


def test_difference_example(oracle_mod):
    g = gold("difference_example.json")
    a = oracle_mod.Bitmap.from_sorted(g["A"])
    b = oracle_mod.Bitmap.from_sorted(g["B"])
    assert a.op(oracle_mod.ANDNOT, b).to_u32().tolist() == g["A_minus_B"]
    # the block masks of the worked example: which values of A meet each block of B
    A = np.array(g["A"])
    m1 = sum(1 << i for i, v in enumerate(A) if v in g["B"][:4])
    m2 = sum(1 << i for i, v in enumerate(A) if v in g["B"][4:])
    assert (m1, m2, m1 | m2) == (g["masks"]["block1"], g["masks"]["block2"], g["masks"]["or"])
    kept = [int(v) for i, v in enumerate(A) if not (g["masks"]["or"] >> i) & 1]
    assert kept == g["A_minus_B"]


def test_dedup_example(oracle_mod):
    g = gold("dedup_example.json")
    a = oracle_mod.Bitmap.from_sorted(g["A"])
    b = oracle_mod.Bitmap.from_sorted(g["B"])
    assert a.op(oracle_mod.OR, b).to_u32().tolist() == g["union"]
    assert a.op(oracle_mod.XOR, b).to_u32().tolist() == g["xor"]


def test_array_bitset_union_example(oracle_mod):
    g = gold("array_bitset_example.json")
    dense = np.arange(200, 200 + 2 * 5000, 2, dtype=np.uint32)  # 5000 values -> bitset
    bs = oracle_mod.Bitmap.from_sorted(dense)
    assert bs.layout()["types"].tolist() == [1]
    arr = oracle_mod.Bitmap.from_sorted(g["array"])
    u = bs.op(oracle_mod.OR, arr)
    lay = u.layout()
    words = lay["payload"].view(np.uint64)
    for v in g["array"]:
        assert (int(words[v >> 6]) >> (v & 63)) & 1
    assert u.card == 5000 + len(g["array"])


def _thr(oracle_mod, values):
    lay = oracle_mod.Bitmap.from_sorted(np.asarray(values, np.uint32)).layout()
    check_canonical(lay)
    return int(lay["types"][0]), int(lay["cards"][0]), lay


def test_type_thresholds(oracle_mod):
    g = gold("type_thresholds.json")
    isolated = np.arange(0, 2 * 4097, 2)
    assert _thr(oracle_mod, isolated[:g["array_max"]])[0] == 0          # 4096 -> array
    assert _thr(oracle_mod, isolated[:g["bitset_min"]])[0] == 1         # 4097 -> bitset
    # c > 4096: 2047 runs -> run container, 2048 runs -> bitset
    def runs_set(nr, c):
        base = c // nr
        lens = [base + (1 if i < c - base * nr else 0) for i in range(nr)]
        out, pos = [], 0
        for L in lens:
            out.extend(range(pos, pos + L))
            pos += L + 1
        assert pos <= 65537
        return out
    t, c, _ = _thr(oracle_mod, runs_set(g["run_max_runs_when_large"], 8000))
    assert (t, c) == (2, 8000)
    t, c, _ = _thr(oracle_mod, runs_set(g["run_max_runs_when_large"] + 1, 8000))
    assert (t, c) == (1, 8000)
    # c <= 4096: runs iff 2r < c
    assert _thr(oracle_mod, runs_set(49, 100))[0] == 2
    assert _thr(oracle_mod, runs_set(50, 100))[0] == 0
    assert _thr(oracle_mod, runs_set(50, 101))[0] == 2
    # full container is one run <0, 65535> (Sec. 2.2)
    t, c, lay = _thr(oracle_mod, np.arange(65536))
    assert (t, c) == (2, 65536)
    assert lay["payload"].view(np.uint16).tolist() == g["full_container_run"]


def random_set(rng, nchunks=3):
    """Small sets with values near word and chunk boundaries, runs, dense blocks."""
    parts = []
    for k in range(nchunks):
        if rng.random() < 0.25:
            continue
        base = k << 16
        kind = rng.integers(0, 5)
        if kind == 0:
            parts.append(base + rng.choice(65536, size=rng.integers(1, 60), replace=False))
        elif kind == 1:
            edges = np.array([0, 1, 62, 63, 64, 65, 127, 128, 4095, 4096, 65534, 65535])
            parts.append(base + rng.choice(edges, size=rng.integers(1, len(edges)), replace=False))
        elif kind == 2:
            s = int(rng.integers(0, 65000))
            parts.append(base + np.arange(s, min(65536, s + int(rng.integers(1, 3000)))))
        elif kind == 3:
            parts.append(base + rng.choice(65536, size=int(rng.integers(4000, 9000)), replace=False))
        else:
            starts = np.sort(rng.choice(65536 // 8, size=int(rng.integers(1, 40)), replace=False)) * 8
            parts.append(base + np.unique(np.concatenate([np.arange(s, min(65536, s + rng.integers(1, 7))) for s in starts])))
    if not parts:
        return np.zeros(0, np.uint32)
    return np.unique(np.concatenate(parts)).astype(np.uint32)


@pytest.mark.parametrize("seed", range(40))
def test_ops_vs_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    a, b = random_set(rng), random_set(rng)
    A, B = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
    assert np.array_equal(A.to_u32(), a)
    assert np.array_equal(decode_layout(A.layout()), a)
    for op in range(4):
        R = A.op(op, B)
        exp = ref_op(op, a, b)
        assert np.array_equal(R.to_u32(), exp), op
        lay = R.layout()
        check_canonical(lay)
        assert np.array_equal(decode_layout(lay), exp)
        assert A.op_card(op, B) == len(exp)


def test_count_identities_and_jaccard(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(20):
        a, b = random_set(rng, 4), random_set(rng, 4)
        A, B = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
        i = A.op_card(0, B)
        assert i == len(np.intersect1d(a, b))
        assert A.op_card(1, B) == len(a) + len(b) - i
        assert A.op_card(2, B) == len(a) - i
        assert A.op_card(3, B) == len(a) + len(b) - 2 * i
        j, ii, uu = A.jaccard(B)
        assert ii == i and uu == len(np.union1d(a, b))
        assert j == (ii / uu if uu else 0.0)
        assert 0.0 <= j <= 1.0


def test_multi_way_fold(oracle_mod):
    rng = np.random.default_rng(11)
    sets = [random_set(rng, 3) for _ in range(6)]
    bms = [oracle_mod.Bitmap.from_sorted(s) for s in sets]
    u = oracle_mod.Bitmap.multi(1, bms)
    exp_u = np.unique(np.concatenate(sets)).astype(np.uint32)
    assert np.array_equal(u.to_u32(), exp_u)
    check_canonical(u.layout())
    common = np.concatenate([np.arange(100, 5000), np.arange(70000, 70100)]).astype(np.uint32)
    sets2 = [np.union1d(s, common).astype(np.uint32) for s in sets]
    bms2 = [oracle_mod.Bitmap.from_sorted(s) for s in sets2]
    inter = oracle_mod.Bitmap.multi(0, bms2)
    exp_i = sets2[0]
    for s in sets2[1:]:
        exp_i = np.intersect1d(exp_i, s)
    assert np.array_equal(inter.to_u32(), exp_i)
    check_canonical(inter.layout())
    assert oracle_mod.Bitmap.multi(1, []).card == 0


def test_invalid_input(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.Bitmap.from_sorted([3, 2])
    with pytest.raises(ValueError):
        oracle_mod.Bitmap.from_sorted([1, 1])


def test_edges(oracle_mod):
    O = oracle_mod
    e = O.Bitmap.from_sorted([])
    assert e.card == 0 and e.n_containers == 0
    top = O.Bitmap.from_sorted([0, 65535, 65536, 0xFFFF0000, 0xFFFFFFFF])
    assert top.layout()["keys"].tolist() == [0, 1, 65535]
    assert np.array_equal(top.to_u32(), np.array([0, 65535, 65536, 0xFFFF0000, 0xFFFFFFFF], np.uint32))
    for op in range(4):
        assert np.array_equal(top.op(op, e).to_u32(), ref_op(op, top.to_u32(), np.zeros(0, np.uint32)))
        assert np.array_equal(e.op(op, top).to_u32(), ref_op(op, np.zeros(0, np.uint32), top.to_u32()))
    a = O.Bitmap.from_sorted(fig1_values())
    assert np.array_equal(a.op(0, a).to_u32(), fig1_values())
    assert np.array_equal(a.op(1, a).to_u32(), fig1_values())
    assert a.op(2, a).card == 0 and a.op(3, a).card == 0
    assert a.op(3, a).n_containers == 0
    j, i, u = e.jaccard(e)
    assert (j, i, u) == (0.0, 0, 0)


def test_plain_workload_canonical(oracle_mod, workloads_mod):
    pool = workloads_mod.plain_pair(1)
    a, b = pool.values(0), pool.values(1)
    A, B = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
    la, lb = A.layout(), B.layout()
    check_canonical(la)
    check_canonical(lb)
    assert len(la["keys"]) == 200 and len(lb["keys"]) == 200
    assert len(np.intersect1d(la["keys"], lb["keys"])) == 100
    # all three container types occur
    assert set(la["types"].tolist()) == {0, 1, 2}
    for op in range(4):
        R = A.op(op, B)
        check_canonical(R.layout())
        assert np.array_equal(R.to_u32(), ref_op(op, a, b))


def test_membership(oracle_mod):
    """Sec. 1 membership on Fig. 1's bitmap (array, runs and bitset chunks),
    at the values the figure describes and their neighbours, then against
    numpy's isin on random sets."""
    bm = oracle_mod.Bitmap.from_sorted(fig1_values())
    probes = np.array([0, 62, 61938, 61939, 63, 2**16 - 1,            # multiples of 62 below 62,000
                       2**16, 2**16 + 99, 2**16 + 100, 2**16 + 101,    # the gap at 2^16 + 100
                       2**16 + 200, 2**16 + 201, 2**16 + 300, 2**16 + 399, 2**16 + 400,
                       2 * 2**16, 2 * 2**16 + 1, 2 * 2**16 + 2, 3 * 2**16 - 2, 3 * 2**16 - 1,
                       3 * 2**16, 0xFFFFFFFF], np.uint32)
    want = [1, 1, 1, 0, 0, 0,
            1, 1, 0, 1,
            1, 0, 1, 1, 0,
            1, 0, 1, 1, 0,
            0, 0]
    assert bm.contains(probes).tolist() == want
    rng = np.random.default_rng(5)
    for _ in range(10):
        a = random_set(rng, 4)
        q = np.concatenate([a[::3], rng.integers(0, 5 * 2**16, 500, dtype=np.uint32),
                            (a[::5] + 1).astype(np.uint32)]).astype(np.uint32)
        A = oracle_mod.Bitmap.from_sorted(a)
        assert np.array_equal(A.contains(q), np.isin(q, a).astype(np.uint8))


def test_cosine(oracle_mod):
    """Sec. 5 "Fast counts": cosine similarity |A n B| / sqrt(|A| |B|),
    against the closed form over numpy's intersection (one correctly rounded
    product, square root and quotient), and its special cases."""
    import math
    rng = np.random.default_rng(17)
    for _ in range(20):
        a, b = random_set(rng, 4), random_set(rng, 4)
        A, B = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
        c, i = A.cosine(B)
        ii = len(np.intersect1d(a, b))
        assert i == ii
        assert c == (ii / math.sqrt(len(a) * len(b)) if len(a) and len(b) else 0.0)
    f = oracle_mod.Bitmap.from_sorted(fig1_values())
    assert f.cosine(f) == (1.0, len(fig1_values()))
    e = oracle_mod.Bitmap.from_sorted([])
    assert f.cosine(e) == (0.0, 0) and e.cosine(e) == (0.0, 0)
    odd = oracle_mod.Bitmap.from_sorted(np.arange(1, 3 * 2**16, 2, dtype=np.uint32))
    assert f.cosine(odd)[1] == len(np.intersect1d(fig1_values(), np.arange(1, 3 * 2**16, 2)))
