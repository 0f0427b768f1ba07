// rb_serial.cu - a portable byte format for one bitmap (index snapshots).
//
// The paper notes that Roaring has a portable serialized form (Sec. 5,
// memory usage) without giving it; this library defines its own, little
// endian, self-describing and canonical:
//
//   0   u32 magic 0x42474252 ("RBGB")     4   u32 version (1)
//   8   u32 n, containers                  12  u32 reserved (0)
//   16  u64 cardinality                    24  u64 payload bytes
//   32  u16 keys[n], strictly increasing
//       u16 runs[n]: number of runs of a run container, else 0
//       u8  types[n] (0 array, 1 bitset, 2 runs), then zero bytes to a
//           4-byte boundary
//       u32 cards[n]
//       payload of each container in key order: array 2c bytes (ascending
//       u16), bitset 8192 bytes (bit v & 63 of u64 word v >> 6), runs 4r
//       bytes ((start, length - 1) u16 pairs ascending)
//
// These are the parts rb_export_layout returns.  Deserialisation checks every
// field (sortedness, cardinalities, payload sizes, maximal runs, the
// canonical type of each container) on the host before anything reaches the
// device, then uploads the library's device image in one copy.
#include <cstring>
#include <vector>

#include "rb_internal.h"

using namespace rbi;

namespace {

constexpr uint32_t MAGIC = 0x42474252u, VERSION = 1;
constexpr uint64_t HEADER = 32;

uint64_t meta_bytes(uint64_t n) { return HEADER + align_up(5 * n, 4) + 4 * n; }

template <class T>
T rd(const uint8_t *p) {
    T x;
    memcpy(&x, p, sizeof x);
    return x;
}
template <class T>
void wr(uint8_t *p, T x) {
    memcpy(p, &x, sizeof x);
}

// cardinality and maximal runs of a container's payload; false if malformed
bool scan_container(uint32_t type, const uint8_t *p, uint64_t bytes, uint32_t card, uint32_t &runs) {
    runs = 0;
    if (type == T_ARRAY) {
        if (card > ARRAY_MAX || bytes != 2ull * card) return false;
        uint32_t prev = 0;
        for (uint32_t i = 0; i < card; i++) {
            const uint32_t v = rd<uint16_t>(p + 2 * i);
            if (i && v <= prev) return false;
            runs += (i == 0 || v != prev + 1);
            prev = v;
        }
        return true;
    }
    if (type == T_BITSET) {
        if (bytes != 8192) return false;
        uint64_t c = 0, carry = 0;
        for (uint32_t w = 0; w < 1024; w++) {
            const uint64_t x = rd<uint64_t>(p + 8 * w);
            c += __builtin_popcountll(x);
            runs += __builtin_popcountll(x & ~((x << 1) | carry));
            carry = x >> 63;
        }
        return c == card;
    }
    if (type == T_RUN) {
        if (bytes % 4 || bytes == 0) return false;
        const uint32_t r = (uint32_t)(bytes / 4);
        uint64_t c = 0;
        int64_t prev_end = -2;   // last value of the previous run
        for (uint32_t k = 0; k < r; k++) {
            const uint32_t s = rd<uint16_t>(p + 4 * k), l = rd<uint16_t>(p + 4 * k + 2);
            if ((int64_t)s <= prev_end + 1 || s + l > 65535) return false;   // sorted, disjoint, maximal
            c += l + 1;
            prev_end = s + l;
        }
        runs = r;
        return c == card;
    }
    return false;
}

}  // namespace

extern "C" {

rb_status rb_serialize(const rb_t *b, uint8_t *buf, uint64_t cap, uint64_t *n_bytes, void *stream) {
    if (!b) return set_err(RB_EINVAL, "rb_serialize: NULL handle");
    uint32_t n = 0;
    uint64_t pay = 0;
    rb_status st = rb_info(b, &n, &pay);
    if (st != RB_OK) return st;
    const uint64_t meta = meta_bytes(n), total = meta + pay;
    if (n_bytes) *n_bytes = total;
    if (!buf) return RB_OK;
    if (cap < total) return set_err(RB_ERANGE, "rb_serialize: capacity %llu below %llu bytes",
                                    (unsigned long long)cap, (unsigned long long)total);
    std::vector<uint16_t> keys(n), runs(n, 0);
    std::vector<uint8_t> types(n);
    std::vector<uint32_t> cards(n);
    std::vector<uint64_t> offs(n + 1);
    st = rb_export_layout(b, keys.data(), types.data(), cards.data(), offs.data(), buf + meta, pay, stream);
    if (st != RB_OK) return st;
    memset(buf, 0, meta);
    wr<uint32_t>(buf, MAGIC);
    wr<uint32_t>(buf + 4, VERSION);
    wr<uint32_t>(buf + 8, n);
    wr<uint64_t>(buf + 16, b->card);
    wr<uint64_t>(buf + 24, pay);
    for (uint32_t i = 0; i < n; i++)
        if (types[i] == T_RUN) runs[i] = (uint16_t)((offs[i + 1] - offs[i]) / 4);
    uint8_t *p = buf + HEADER;
    if (n) {
        memcpy(p, keys.data(), 2ull * n);
        memcpy(p + 2ull * n, runs.data(), 2ull * n);
        memcpy(p + 4ull * n, types.data(), n);
        memcpy(p + align_up(5ull * n, 4), cards.data(), 4ull * n);
    }
    return RB_OK;
}

rb_status rb_deserialize(const uint8_t *buf, uint64_t len, void *stream, rb_t **out) {
    clear_stale_error();
    if (!out) return set_err(RB_EINVAL, "rb_deserialize: out is NULL");
    *out = nullptr;
    if (!buf || len < HEADER) return set_err(RB_EINVAL, "rb_deserialize: buffer shorter than the header");
    if (rd<uint32_t>(buf) != MAGIC || rd<uint32_t>(buf + 4) != VERSION)
        return set_err(RB_EINVAL, "rb_deserialize: bad magic or version");
    const uint32_t n = rd<uint32_t>(buf + 8);
    const uint64_t card = rd<uint64_t>(buf + 16), pay = rd<uint64_t>(buf + 24);
    if (n > 65536 || rd<uint32_t>(buf + 12) != 0) return set_err(RB_EINVAL, "rb_deserialize: bad header");
    const uint64_t meta = meta_bytes(n);
    if (len < meta || len - meta != pay) return set_err(RB_EINVAL, "rb_deserialize: length does not match the header");
    const uint8_t *kp = buf + HEADER, *rp = kp + 2ull * n, *tp = kp + 4ull * n, *cp = kp + align_up(5ull * n, 4);
    const uint8_t *pp = buf + meta;
    // validate and lay out the device image: keys | descs | word payload | bitsets
    std::vector<uint64_t> descs(n);
    std::vector<uint64_t> src(n);
    uint64_t words = 0, bits = 0, sum = 0, at = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t key = rd<uint16_t>(kp + 2ull * i), type = tp[i], c = rd<uint32_t>(cp + 4ull * i);
        if (i && key <= rd<uint16_t>(kp + 2ull * (i - 1))) return set_err(RB_EINVAL, "rb_deserialize: keys not increasing");
        if (c == 0 || c > 65536 || type > T_RUN) return set_err(RB_EINVAL, "rb_deserialize: bad container %u", i);
        const uint32_t r = rd<uint16_t>(rp + 2ull * i);
        if ((type == T_RUN) != (r != 0)) return set_err(RB_EINVAL, "rb_deserialize: bad run count %u", i);
        const uint64_t bytes = payload_bytes(type, c, r);
        if (at + bytes > pay) return set_err(RB_EINVAL, "rb_deserialize: payload too short");
        uint32_t runs = 0;
        if (!scan_container(type, pp + at, bytes, c, runs))
            return set_err(RB_EINVAL, "rb_deserialize: malformed container %u", i);
        if (canon_type(c, runs) != type)
            return set_err(RB_EINVAL, "rb_deserialize: container %u is not in canonical form", i);
        src[i] = at;
        at += bytes;
        sum += c;
        if (type == T_BITSET) {
            descs[i] = mk_desc(c, T_BITSET, 0, bits);   // relative to the bitset region for now
            bits += 8192;
        } else {
            descs[i] = mk_desc(c, type, type == T_RUN ? runs : 0, words);
            words += word_alloc_bytes(type, c, runs);
        }
    }
    if (at != pay || sum != card) return set_err(RB_EINVAL, "rb_deserialize: sizes do not add up");
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t descs_off = align_up(2ull * n, 256), words_off = align_up(descs_off + 8ull * n, 256);
    const uint64_t bits_off = align_up(words_off + words, 256), total = std::max<uint64_t>(bits_off + bits, 16);
    if (total >= MAX_OFFSET) return set_err(RB_ERANGE, "rb_deserialize: bitmap above the 128 GiB descriptor reach");
    uint8_t *img = (uint8_t *)pinned_scratch(total);
    if (!img) return set_err(RB_ENOMEM, "pinned staging allocation failed");
    memset(img, 0, total);
    uint32_t nbits = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t d = descs[i];
        const uint32_t type = d_type(d), c = d_card(d), r = d_runs(d);
        const uint64_t off = (type == T_BITSET ? bits_off : words_off) + d_off(d);
        memcpy(img + off, pp + src[i], payload_bytes(type, c, r));
        descs[i] = mk_desc(c, type, r, off);
        nbits += type == T_BITSET;
    }
    if (n) {
        memcpy(img, kp, 2ull * n);
        memcpy(img + descs_off, descs.data(), 8ull * n);
    }
    rb *h = handle_new();
    h->arena = arena_new(total, s);
    if (!h->arena) { delete h; return RB_ENOMEM; }
    h->base = (uint8_t *)h->arena->ptr;
    h->keys = (uint16_t *)h->base;
    h->descs = (uint64_t *)(h->base + descs_off);
    h->n = n;
    h->card = card;
    h->word_bytes = words;
    h->n_bitsets = nbits;
    cudaError_t e = cudaMemcpyAsync(h->base, img, total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        rb_free(h);
        return cuda_err(e, "rb_deserialize upload");
    }
    *out = h;
    return RB_OK;
}

}  // extern "C"
