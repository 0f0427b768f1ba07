"""The threshold cases (tests/threshold_cases.py) on the CPU: every case's
result, computed by the oracle, is exactly its target set, and the target
sits on the type boundary it is named for (Sec. 1's constraints).  This pins
the cases themselves, so that the GPU tests that route them through every
kernel path test what they claim to."""
import numpy as np

from threshold_cases import TARGETS, canon, cases, runs_of, with_keys


def test_targets_sit_on_the_boundaries():
    for name, c, r, _, _ in TARGETS:
        t = canon(c, r)
        if "2r=c-" in name:
            assert c <= 4096 and 2 * r < c and t == 2, name
        elif "2r=c+" in name or name.endswith("2r=c"):
            assert c <= 4096 and 2 * r >= c and t == 0, name
        if "r=2047" in name:
            assert c > 4096 and t == 2, name
        if "r=2048" in name:
            assert c > 4096 and t == 1, name
    names = [n for n, *_ in TARGETS]
    assert "c=4096 array" in names and "c=4097 bitset" in names


def test_every_case_yields_its_target(oracle_mod):
    cs = with_keys(cases(), lambda i: 65535 if i % 5 == 1 else (i * 977) % 65536)
    seen_types = set()
    for name, op, a, b, T in cs:
        A, B = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
        R = A.op(op, B)
        assert np.array_equal(R.to_u32(), T), name
        lay = R.layout()
        assert len(lay["keys"]) == 1, name
        low = T & 0xFFFF
        ty = int(lay["types"][0])
        assert ty == canon(len(low), runs_of(low)), name
        seen_types.add(ty)
        A.close(), B.close(), R.close()
    assert seen_types == {0, 1, 2}


def test_input_classes_cover_every_path(oracle_mod):
    """The inputs reach every container-pair path: array pairs of at most 64,
    254 and 1022 values and larger ones, bitset pairs, and run inputs."""
    cs = cases()
    sizes, kinds = [], set()
    for name, op, a, b, T in cs:
        if len(a) == 0 or len(b) == 0:
            continue
        A, B = oracle_mod.Bitmap.from_sorted(a), oracle_mod.Bitmap.from_sorted(b)
        ta, tb = int(A.layout()["types"][0]), int(B.layout()["types"][0])
        kinds.add((ta, tb))
        if ta == 0 and tb == 0:
            sizes.append(len(a) + len(b))
        A.close(), B.close()
    sizes = np.array(sizes)
    assert np.any(sizes <= 64) and np.any((sizes > 64) & (sizes <= 254))
    assert np.any((sizes > 254) & (sizes <= 1022)) and np.any(sizes > 1022)
    assert (1, 1) in kinds and any(2 in k for k in kinds) and any(0 in k and 1 in k for k in kinds)
