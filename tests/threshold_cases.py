"""Container pairs whose operation OUTPUT lands exactly on the canonical-type
boundaries (Sec. 1's constraints, read as "smallest of array 2c B, bitset
8 KB, runs 4r B" with ties to array / bitset):

  c <= 4096:  runs iff 2r < c     -> targets 2r = c, 2r = c - 1, 2r = c + 1
  c  = 4096 / 4097                 -> array (or runs) / bitset (or runs)
  c  > 4096:  runs iff r <= 2047   -> targets r = 2047 / 2048
  the full chunk <0,65535>, and the values 0 and 65535 at the chunk edges.

Each target T (c values, r maximal runs, in one chunk) is produced by every
op from inputs built around it:

  AND     A = T + XA,            B = T + XB
  OR      A = T[0::2],           B = T[1::2]        (or A = T, B = T[1::3])
  ANDNOT  A = T + X,             B = X + Y
  XOR     A = T[0::2] + S,       B = T[1::2] + S

where X, XA, XB, Y, S are disjoint sets of isolated values placed in T's
gaps.  The sizes of the targets and of the padding pick the path that
computes the pair (the limits of the container-pair kernels): up to 64
values in both inputs one lane merges or sweeps, up to 254 a group of 8
lanes, up to 1022 the whole warp, anything larger or with a bitset the
heavy kernel (bit probes into a list, or 8 KB tiles).

Only numpy is used here: the cases are inputs, and the expected results
come from the oracle.
"""
import numpy as np

# (name, c, r, small padding, large padding): the padding sizes pick the
# input sizes (and so the kernel path) for AND / ANDNOT / XOR
TARGETS = [
    # one lane (both inputs at most 64 values)
    ("lane 2r=c", 8, 4, 2, None),
    ("lane 2r=c-1", 9, 4, 2, None),
    ("lane 2r=c+1", 9, 5, 2, None),
    ("lane 2r=c-2", 12, 5, 2, None),
    ("lane single", 1, 1, 2, None),
    # a group of 8 lanes (at most 254)
    ("group 2r=c", 100, 50, 4, None),
    ("group 2r=c-1", 101, 50, 4, None),
    ("group 2r=c+1", 99, 50, 4, None),
    # the whole warp (at most 1022)
    ("warp 2r=c", 400, 200, 8, None),
    ("warp 2r=c-1", 401, 200, 8, None),
    ("warp 2r=c+1", 399, 200, 8, None),
    # the heavy kernel: array inputs (bit probes, list emit) with the small
    # padding, bitset inputs (tiles) with the large one
    ("heavy 2r=c", 4000, 2000, 8, 600),
    ("heavy 2r=c-1", 4001, 2000, 8, 600),
    ("heavy 2r=c+1", 3999, 2000, 8, 600),
    ("c=4096 array", 4096, 2048, 8, 600),
    ("c=4096 runs", 4096, 2047, 8, 600),
    ("c=4097 bitset", 4097, 2048, 8, 600),
    ("c=4097 runs", 4097, 2047, 8, 600),
    ("c>4096 r=2047", 6000, 2047, 8, 600),
    ("c>4096 r=2048", 6000, 2048, 8, 600),
    ("dense r=2047", 30000, 2047, 8, 600),
    ("dense r=2048", 30000, 2048, 8, 600),
    ("c=65535 r=2", 65535, 2, None, None),
]


def canon(c, r):
    """0 array, 1 bitset, 2 runs."""
    if c <= 4096:
        return 2 if 2 * r < c else 0
    return 2 if r <= 2047 else 1


def target_chunk(rng, c, r, gap_min=3):
    """c values of [0, 65536) in exactly r maximal runs, from 0 to 65535
    (both edge values present when r > 1; one run ends at 65535), inner gaps
    of at least gap_min."""
    if r == 1:                            # one run ending at 65535
        return np.arange(65536 - c, 65536, dtype=np.uint32)
    if c == 65535 and r == 2:             # everything but one value
        hole = int(rng.integers(1, 65535))
        return np.delete(np.arange(65536, dtype=np.uint32), hole)
    lens = np.diff(np.concatenate([[0], np.sort(rng.choice(np.arange(1, c), r - 1, replace=False)), [c]]))
    free = 65536 - c - gap_min * (r - 1)
    assert free >= 0, (c, r)
    cuts = np.sort(rng.integers(0, free + 1, r - 2)) if r > 2 else np.zeros(0, np.int64)
    extra = np.diff(np.concatenate([[0], cuts, [free]]))
    gaps = gap_min + extra
    out, pos = [], 0
    for i in range(r):
        out.append(np.arange(pos, pos + lens[i]))
        pos += lens[i] + (gaps[i] if i < r - 1 else 0)
    v = np.concatenate(out).astype(np.uint32)
    assert v[0] == 0 and v[-1] == 65535 and len(v) == c
    return v


def isolated(rng, taken, n):
    """n values of [0, 65536), none in `taken` or next to a value of it,
    nor next to each other."""
    if n == 0:
        return np.zeros(0, np.uint32)
    mark = np.zeros(65536 + 2, bool)
    t = taken.astype(np.int64)
    mark[t] = True
    mark[t + 1] = True
    mark[np.maximum(t - 1, 0)] = True
    cand = np.nonzero(~mark[:65536])[0]
    cand = cand[cand % 2 == 0]            # no two picks adjacent
    assert len(cand) >= n, (len(cand), n)
    return np.sort(rng.choice(cand, n, replace=False)).astype(np.uint32)


def u(*parts):
    return np.unique(np.concatenate(parts)).astype(np.uint32)


def cases(seed=1709):
    """(name, op, a_low, b_low, T): low 16-bit values of one chunk each
    (T is the expected result)."""
    rng = np.random.default_rng(seed)
    out = []
    for name, c, r, pad_s, pad_l in TARGETS:
        T = target_chunk(rng, c, r)
        ev, od = T[0::2], T[1::2]
        out.append((name + " | OR halves", 1, ev, od, T))
        out.append((name + " | OR whole+part", 1, T, T[1::3], T))
        for pad, tag in ((pad_s, "small pad"), (pad_l, "large pad")):
            if pad is None:
                continue
            X = isolated(rng, T, 3 * pad)
            XA, XB, Y = X[0::3], X[1::3], X[2::3]
            out.append((f"{name} | AND {tag}", 0, u(T, XA), u(T, XB), T))
            out.append((f"{name} | ANDNOT {tag}", 2, u(T, XA), u(XA, Y), T))
            out.append((f"{name} | XOR {tag}", 3, u(ev, XA), u(od, XA), T))
    # the full chunk as one run <0,65535>, and its complement pieces
    F = np.arange(65536, dtype=np.uint32)
    out.append(("full | OR evens odds", 1, F[0::2], F[1::2], F))
    out.append(("full | XOR evens odds", 3, F[0::2], F[1::2], F))
    out.append(("full | AND full full", 0, F, F, F))
    out.append(("full | OR halves", 1, F[:32768], F[32768:], F))
    out.append(("full | OR runs", 1, u(F[:40000]), u(F[30000:]), F))
    # only the edge values
    E = np.array([0, 65535], np.uint32)
    out.append(("edges | AND", 0, u(E, [5, 9]), u(E, [7]), E))
    out.append(("edges | OR", 1, E[:1], E[1:], E))
    out.append(("edges | XOR", 3, np.array([0, 3, 65535], np.uint32), np.array([3], np.uint32), E))
    return out


def with_keys(cases_, key_of):
    """Full uint32 value arrays: the chunk of case i at key key_of(i)."""
    res = []
    for i, (name, op, a, b, T) in enumerate(cases_):
        k = np.uint32(key_of(i)) << np.uint32(16)
        res.append((name, op, (k | a).astype(np.uint32), (k | b).astype(np.uint32), (k | T).astype(np.uint32)))
    return res


def runs_of(v):
    v = np.asarray(v, np.int64)
    return 0 if len(v) == 0 else 1 + int(np.count_nonzero(np.diff(v) != 1))
