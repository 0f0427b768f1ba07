"""Multi-way AND / OR paths of the kernel that folds each output key in one
8 KB tile per warp, each reached on purpose and compared with the oracle's
layout bit for bit (Sec. 5 "Wide unions" computes the union of many sets; the
intersection is its dual):

- folds in place: AND with an array that is not the key's first container,
  AND and OR with run containers (runs that start at 0, end at 65535, cover
  the whole chunk), bitsets combined last;
- run results written without scratch (canonical type runs after a fold);
- a lane key whose arrays do not fit the staging tile (folded instead);
- tiles whose lane keys need several staging rounds (32 keys of about 600
  values in play each).

Each bitmap is built key by key with the container kind chosen for that
key, so the member order within a key (which container a fold starts from)
is fixed by construction."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FIELDS = ("keys", "types", "cards", "offs", "payload")


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


def array_of(rng, c):
    return np.sort(rng.choice(65536, size=c, replace=False)).astype(np.uint32)


def bitset_of(rng, c):
    assert c > 4096
    return array_of(rng, c)


def runs_of(rng, nr, lo=2, hi=40, start0=False, end65535=False):
    """nr maximal runs (gaps of at least 2) with lengths in [lo, hi)."""
    lens = rng.integers(lo, hi, size=nr)
    gaps = rng.integers(2, max(3, (65536 - int(lens.sum())) // max(nr, 1)), size=nr)
    out, pos = [], 0 if start0 else int(gaps[0])
    for i in range(nr):
        out.append(np.arange(pos, min(65536, pos + int(lens[i]))))
        pos += int(lens[i]) + int(gaps[(i + 1) % nr])
        if pos >= 65536:
            break
    v = np.unique(np.concatenate(out)).astype(np.uint32)
    if end65535:
        v = np.union1d(v, np.arange(65500, 65536)).astype(np.uint32)
    return v


def bitmap_values(chunks):
    """uint32 values of a bitmap given {key: low 16-bit values}."""
    parts = [(np.uint32(k) << np.uint32(16)) | v.astype(np.uint32) for k, v in sorted(chunks.items()) if len(v)]
    return np.concatenate(parts).astype(np.uint32) if parts else np.zeros(0, np.uint32)


def check(rb, oracle_mod, op, members, ctx):
    G = [rb.Bitmap.from_sorted(v) for v in members]
    O = [oracle_mod.Bitmap.from_sorted(v) for v in members]
    exp = oracle_mod.Bitmap.multi(op, O)
    m, card = rb.multi_op(op, G)
    assert card == exp.card, ctx
    assert_layout_eq(m.layout(), exp.layout(), ctx)
    _, c0 = rb.multi_op(op, G, count_only=True)
    assert c0 == exp.card, ctx
    return exp


def test_in_place_folds_and_direct_run_emit(rb, oracle_mod):
    """One key per combination; member 0's container is the one a fold
    starts from."""
    rng = np.random.default_rng(1709)
    full = np.arange(65536, dtype=np.uint32)
    combos = [
        # AND: runs first, then an array (in-place AND with an array), a bitset
        (0, ["runs_big", "array_big", "bitset"]),
        # AND: array first, then runs (in-place AND with runs: gaps cleared)
        (0, ["array_big", "runs_big", "bitset"]),
        # AND of runs only: the result stays runs (written without scratch)
        (0, ["runs_edge", "runs_wide"]),
        (0, ["full", "runs_edge", "bitset_dense"]),
        # OR: runs (set in place), arrays, bitsets
        (1, ["runs_big", "array_big", "bitset"]),
        (1, ["runs_edge", "runs_wide"]),
        (1, ["runs_big", "array_small", "runs_wide"]),
        (1, ["full", "array_big"]),
    ]

    def make(kind):
        if kind == "runs_big":
            return runs_of(rng, 300, 4, 120)
        if kind == "runs_wide":
            return runs_of(rng, 40, 500, 1500)
        if kind == "runs_edge":
            return runs_of(rng, 60, 100, 400, start0=True, end65535=True)
        if kind == "array_big":
            return array_of(rng, 3000)
        if kind == "array_small":
            return array_of(rng, 40)
        if kind == "bitset":
            return bitset_of(rng, 30000)
        if kind == "bitset_dense":
            return bitset_of(rng, 60000)
        return full

    for op in (0, 1):
        sel = [c for c in combos if c[0] == op]
        k = max(len(kinds) for _, kinds in sel)
        chunks = [dict() for _ in range(k)]
        for key, (_, kinds) in enumerate(sel):
            for i in range(k):
                # AND needs every member at the key: extra members hold the
                # whole chunk; OR leaves them out
                kind = kinds[i] if i < len(kinds) else ("full" if op == 0 else None)
                if kind is not None:
                    chunks[i][3 * key + 1] = make(kind)
        exp = check(rb, oracle_mod, op, [bitmap_values(c) for c in chunks], f"folds op {op}")
        assert 2 in set(exp.layout()["types"].tolist()), "no run result: the direct run emit is not reached"


def test_lane_key_too_large_for_the_tile(rb, oracle_mod):
    """AND keys whose smallest array is small (a lane candidate) but whose
    arrays in all take more than the 8 KB tile: folded by the warp, next to
    keys that the lanes merge."""
    rng = np.random.default_rng(7)
    chunks = [dict(), dict(), dict()]
    for key in range(0, 64):
        if key % 4 == 0:   # 100 + 4096 + 4096 values: 4,146 words
            common = array_of(rng, 100)
            chunks[0][key] = common
            chunks[1][key] = np.union1d(common[::2], array_of(rng, 4096))[:4096].astype(np.uint32)
            chunks[2][key] = np.union1d(common[1::3], array_of(rng, 4096))[:4096].astype(np.uint32)
        else:
            base = array_of(rng, 300)
            for i in range(3):
                chunks[i][key] = np.union1d(base[::2 + i], array_of(rng, 50)).astype(np.uint32)
    vals = [bitmap_values(c) for c in chunks]
    check(rb, oracle_mod, 0, vals, "AND lane overflow")
    check(rb, oracle_mod, 1, vals, "OR of the same")


@pytest.mark.parametrize("op", [0, 1])
def test_staging_rounds(rb, oracle_mod, op):
    """Every key of several tiles is a lane key with about 600 values in play
    (4 members of about 150): a tile's keys take about 9,600 words, several
    staging rounds of the 2,048-word tile."""
    rng = np.random.default_rng(11 + op)
    chunks = [dict() for _ in range(4)]
    for key in range(0, 200):
        shared = array_of(rng, 120)
        for i in range(4):
            own = array_of(rng, 40)
            chunks[i][key] = np.union1d(shared if op == 0 else shared[i::4], own).astype(np.uint32)
    check(rb, oracle_mod, op, [bitmap_values(c) for c in chunks], f"staging rounds op {op}")
