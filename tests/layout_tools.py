"""Test helpers: decode an exported Roaring layout and check canonical form.

Written independently of both the oracle and the CUDA library, from the
format definition: per container a u16 key, a u8 type (0 array, 1 bitset,
2 runs), a u32 cardinality and payload bytes (array: ascending u16; bitset:
1024 little-endian u64 words, bit v & 63 of word v >> 6; runs: (start,
length - 1) u16 pairs), concatenated in key order with offsets offs[n + 1].
"""
import numpy as np

TYPE_NAMES = {0: "array", 1: "bitset", 2: "run"}


def decode_container(t, payload):
    if t == 0:
        return payload.view(np.uint16).astype(np.uint32)
    if t == 1:
        words = payload.view(np.uint64)
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")
        return np.nonzero(bits)[0].astype(np.uint32)
    if t == 2:
        pairs = payload.view(np.uint16).reshape(-1, 2).astype(np.uint32)
        if len(pairs) == 0:
            return np.zeros(0, np.uint32)
        return np.concatenate([np.arange(s, s + l + 1, dtype=np.uint32) for s, l in pairs])
    raise AssertionError(f"bad type {t}")


def decode_layout(lay):
    parts = []
    for i in range(len(lay["keys"])):
        o0, o1 = int(lay["offs"][i]), int(lay["offs"][i + 1])
        low = decode_container(int(lay["types"][i]), lay["payload"][o0:o1])
        parts.append((np.uint32(lay["keys"][i]) << np.uint32(16)) | low)
    if not parts:
        return np.zeros(0, np.uint32)
    return np.concatenate(parts).astype(np.uint32)


def check_canonical(lay):
    """Assert the paper's container constraints (Sec. 1) and basic well-formedness."""
    keys = lay["keys"].astype(np.int64)
    assert np.all(np.diff(keys) > 0), "keys not strictly increasing"
    for i in range(len(keys)):
        t = int(lay["types"][i])
        c = int(lay["cards"][i])
        o0, o1 = int(lay["offs"][i]), int(lay["offs"][i + 1])
        pl = lay["payload"][o0:o1]
        low = decode_container(t, pl)
        assert c >= 1, "empty container"
        assert len(low) == c, f"card {c} != recount {len(low)}"
        assert np.all(np.diff(low.astype(np.int64)) > 0), "values not strictly increasing"
        r = 1 + int(np.count_nonzero(np.diff(low.astype(np.int64)) != 1))
        if t == 0:
            assert c <= 4096 and o1 - o0 == 2 * c
            assert not (2 * r < c), "array that should be runs"
        elif t == 1:
            assert c >= 4097 and o1 - o0 == 8192
            assert r > 2047, "bitset that should be runs"
        else:
            pairs = pl.view(np.uint16).reshape(-1, 2).astype(np.int64)
            assert len(pairs) == r, "runs not maximal"
            assert np.all(pairs[:, 0] + pairs[:, 1] <= 65535)
            if len(pairs) > 1:
                assert np.all(pairs[1:, 0] > pairs[:-1, 0] + pairs[:-1, 1] + 1), "runs adjacent/overlapping"
            if c > 4096:
                assert r <= 2047
            else:
                assert 2 * r < c


def image_from_layout(lay):
    """The portable byte image of a bitmap (the format include/rb.h
    documents for rb_serialize), composed from an exported layout."""
    import struct
    keys, types, cards, offs, payload = lay["keys"], lay["types"], lay["cards"], lay["offs"], lay["payload"]
    n = len(keys)
    runs = np.zeros(n, np.uint16)
    for i in range(n):
        if types[i] == 2:
            runs[i] = (int(offs[i + 1]) - int(offs[i])) // 4
    head = struct.pack("<IIIIQQ", 0x42474252, 1, n, 0, int(cards.astype(np.uint64).sum()), len(payload))
    body = keys.astype("<u2").tobytes() + runs.astype("<u2").tobytes() + types.astype(np.uint8).tobytes()
    body += b"\0" * ((-len(body)) % 4)
    body += cards.astype("<u4").tobytes()
    return head + body + payload.tobytes()
