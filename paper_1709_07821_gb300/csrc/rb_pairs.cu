// rb_pairs.cu - pairwise operations: key merge, container-pair kernels,
// canonical compaction, batches, plans (CUDA graphs) and the autotuner.
//
// Work decomposition.  Every query (a op b) owns a range of "slots", cut into
// tiles of 32 that the warps of a persistent kernel steal from one atomic
// counter.  Two slot modes:
//   merge  - slot d is element d of the merge of both key lists (a's key first
//            on a tie).  A tile finds where its 32 elements start with a
//            cooperative 32-ary merge-path search and reads both key windows
//            with one coalesced load each.  Used for OR/XOR always and for
//            AND/ANDNOT/counts when the key counts are within a factor of 8.
//   driver - slot i is key i of one input (the smaller one for AND and
//            counts, a for ANDNOT), and each lane binary-searches the other
//            key list.  Used for skewed AND/ANDNOT/count queries.
// A key present in both inputs becomes one container pair (Sec. 1: containers
// are matched by their 16-bit key).  Output positions keep the result's key
// order: the merged index for OR/XOR (b's copy of a shared key only marks its
// position empty), a's key index for AND/ANDNOT.  Every position of a query's
// output range is written exactly once, so compaction only drops empties.
//
// Kernels.  k_lean (high occupancy, small shared buffers) does the key merge
// of a tile, copies the tile's unmatched array and run containers with the
// whole warp, and queues its container pairs.  Small pairs go to the
// small-pair queue that k_small drains 32 at a time: one pair per lane (small
// array merges, run sweeps) or by groups of 8 lanes or the whole warp in turn
// (array pairs up to 1024 values).  Pairs with a bitset or more values go to
// a deferred queue that k_heavy (one warp per pair, two 8 KB shared tiles per
// warp, bitsets moved by bulk copies) drains.  k_compact then drops the empty
// results of every query.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rb_device.cuh"

using namespace rbi;
using namespace rbd;

namespace {

constexpr uint32_t F_COUNT = 1, F_MERGE = 2;
enum : uint32_t { K_NONE = 0, K_EMPTY = 1, K_PAIR = 2, K_COPY_A = 3, K_COPY_B = 4 };
constexpr int LEAN_THREADS = 128;
// resident k_lean CTAs per SM (a bound of 64 registers per thread)
constexpr uint32_t LEAN_CTAS_MAX = 8;
constexpr uint32_t KEY_END = 0x10000u;   // past-the-end key sentinel
// algorithmic bytes of a container's key and metadata (key 2, type 1,
// cardinality 4, payload offset 8), whatever the layout packs them into,
// and of a count-only result
constexpr uint32_t META_BYTES = 15, COUNT_BYTES = 8;

struct PairDev {
    uint32_t a, b, op, flags;
    uint32_t n_slots, n_pos;
    unsigned long long pos_base;
};

struct PairStats {
    unsigned long long card;      // output cardinality (count-only: |a n b|)
    unsigned long long words;     // word-region bytes of the output
    unsigned long long in_bytes;  // algorithmic input bytes read
    unsigned int n_out, pad0, nbits, pad1;
};

struct Deferred {
    unsigned long long da, db;
    uint32_t p, pos;
    uint32_t kind_key, pad;
};

// a container pair for the small-pair kernel (one-lane, 8-lane group or
// warp merges and run sweeps)
struct Item {
    unsigned long long da, db;
    uint32_t p, pos;
    uint32_t info;   // key | kind << 16 | mode << 20
    uint32_t pad;
};

// Run state in device memory.  The small-pair queue small[0, small_cap)
// holds the one-lane items from index 0 up (small_n1 of them) and the
// group and warp items from the top down (small_n2); the small-pair kernel
// checks small_n1 + small_n2 <= small_cap before it reads any item.
struct ExecState {
    uint8_t *arena;
    uint16_t *keys;
    uint64_t *descs;
    Deferred *defer;
    Item *small;
    unsigned long long words_off, words_cap, bits_off, bits_cap;
    unsigned long long words_used, bits_used, work, hwork;
    unsigned long long defer_cap, defer_n;
    unsigned long long small_cap, small_n1, small_n2, swork1, swork2;
    unsigned long long lean_bytes, heavy_bytes, small_bytes;
    unsigned long long cwork;   // k_compact's query counter
    unsigned int status;
    unsigned int wchunk;        // bytes of a per-warp word chunk (a power of two)
};

// both input views of a query, so that a kernel reads them without first
// reading the query's pool indexes
struct QViews {
    BmView a, b;
};

struct PairParams {
    const BmView *pool;
    const PairDev *pairs;
    const QViews *qv;
    const unsigned long long *tile_base;
    PairStats *stats;
    ExecState *es;
    unsigned long long n_tiles;
    uint32_t n_pairs;
    uint32_t small_iv;
    uint32_t prefetch;   // payload lines hinted into L2 per queued container
    uint32_t chunk;      // consecutive tiles a warp takes at once
};

// ------------------------------------------------------------ allocation

__device__ __forceinline__ uint64_t alloc_words_warp(ExecState *es, uint32_t bytes, uint32_t lane) {
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&es->words_used, (unsigned long long)bytes);
    old = __shfl_sync(FULL, old, 0);
    if (old + bytes > es->words_cap) {
        if (lane == 0) atomicOr(&es->status, 1u);
        return ALLOC_FAIL;
    }
    return es->words_off + old;
}

__device__ __forceinline__ uint64_t alloc_bitset_warp(ExecState *es, uint32_t lane) {
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&es->bits_used, 8192ull);
    old = __shfl_sync(FULL, old, 0);
    if (old + 8192ull > es->bits_cap) {
        if (lane == 0) atomicOr(&es->status, 1u);
        return ALLOC_FAIL;
    }
    return es->bits_off + old;
}

// Word-region allocation for k_lean: each warp takes a chunk of es->wchunk
// bytes at a time from the shared counter and hands it out itself (state in
// shared memory, wa[0] = next free offset, wa[1] = end of the warp's chunk;
// wa[2], wa[3] gather the current query's cardinality and word bytes);
// requests above 1/8 of a chunk go to the counter directly.  A chunk is
// abandoned only when a request of at most 1/8 of a chunk does not fit, so at
// most 1/8 of the chunked bytes plus one chunk per warp go unused; the arena
// adds that much slack.  The chunk is sized per plan (word_chunk): a batch
// with tens of GB of results refills from the one counter millions of times
// with small chunks, and those same-address atomics serialise.
// Returns the offset within the word region (warp-uniform), or ALLOC_FAIL
// after flagging the overflow.
constexpr uint32_t WCHUNK_MIN = 16384;
constexpr uint32_t WCHUNK_MAX = 131072;
__device__ __forceinline__ uint64_t lean_alloc(ExecState *es, unsigned long long *wa, uint32_t bytes,
                                               uint32_t lane) {
    unsigned long long r = 0;
    if (lane == 0) {
        const unsigned long long cur = wa[0], end = wa[1];
        if (cur + bytes <= end) {
            r = cur;
            wa[0] = cur + bytes;
        } else {
            const uint32_t wchunk = es->wchunk;
            if (bytes > (wchunk >> 3)) {
                r = atomicAdd(&es->words_used, (unsigned long long)bytes);
                if (r + bytes > es->words_cap) r = ALLOC_FAIL;
            } else {
                r = atomicAdd(&es->words_used, (unsigned long long)wchunk);
                if (r + wchunk > es->words_cap) {
                    r = ALLOC_FAIL;
                    wa[0] = wa[1] = 0;
                } else {
                    wa[0] = r + bytes;
                    wa[1] = r + wchunk;
                }
            }
        }
        if (r == ALLOC_FAIL) atomicOr(&es->status, 1u);
    }
    return __shfl_sync(FULL, r, 0);
}

// The same scheme for k_heavy, whose chunk state is warp-uniform registers;
// returns the absolute arena offset, or ALLOC_FAIL after flagging overflow.
struct WChunk {
    unsigned long long cur, end;
};
__device__ __forceinline__ uint64_t chunk_alloc_words(ExecState *es, WChunk &w, uint32_t bytes, uint32_t lane) {
    if (w.cur + bytes <= w.end) {
        const uint64_t r = w.cur;
        w.cur += bytes;
        return es->words_off + r;
    }
    const uint32_t wchunk = es->wchunk;
    const bool direct = bytes > (wchunk >> 3);
    const uint32_t take = direct ? bytes : wchunk;
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&es->words_used, (unsigned long long)take);
    old = __shfl_sync(FULL, old, 0);
    if (old + take > es->words_cap) {
        if (lane == 0) atomicOr(&es->status, 1u);
        if (!direct) w.cur = w.end = 0;
        return ALLOC_FAIL;
    }
    if (!direct) {
        w.cur = old + bytes;
        w.end = old + wchunk;
    }
    return es->words_off + old;
}

// ------------------------------------------------------------ warp paths

// nw 4-byte words from S to D by the warp, 8 loads per lane in flight
// before their stores (the compiler may not move a load above a store that
// could alias it, so a plain loop would wait one memory latency per 128 B)
__device__ __forceinline__ void warp_copy_words(uint32_t *D, const uint32_t *S, uint32_t nw, uint32_t lane) {
    for (uint32_t g0 = 0; g0 < nw; g0 += 256) {
        uint32_t v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t g = g0 + 32u * k + lane;
            v[k] = g < nw ? __ldg(S + g) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t g = g0 + 32u * k + lane;
            if (g < nw) D[g] = v[k];
        }
    }
}

__device__ __noinline__ uint64_t warp_copy(ExecState *es, const CRef &x, uint32_t lane) {
    if (x.type == T_BITSET) {
        uint64_t off = alloc_bitset_warp(es, lane);
        if (off == ALLOC_FAIL) return DESC_EMPTY;
        const ulonglong2 *S = reinterpret_cast<const ulonglong2 *>(x.p);
        ulonglong2 *D = reinterpret_cast<ulonglong2 *>(es->arena + off);
        ulonglong2 v[16];
#pragma unroll
        for (int k = 0; k < 16; k++) v[k] = __ldg(S + 32 * k + lane);
#pragma unroll
        for (int k = 0; k < 16; k++) D[32 * k + lane] = v[k];
        return mk_desc(x.card, T_BITSET, 0, off);
    }
    uint32_t bytes = word_alloc_bytes(x.type, x.card, x.runs);
    uint64_t off = alloc_words_warp(es, bytes, lane);
    if (off == ALLOC_FAIL) return DESC_EMPTY;
    warp_copy_words(reinterpret_cast<uint32_t *>(es->arena + off), reinterpret_cast<const uint32_t *>(x.p), bytes / 4,
                    lane);
    return mk_desc(x.card, x.type, x.type == T_RUN ? x.runs : 0, off);
}

// a op b for one container pair whose result is a subset of an array (AND
// with an array operand, ANDNOT with an array first), by the whole warp:
// each value of the array is tested against the other container (Sec. 3.2
// bit tests; a bitset is read in place, an array or run container is first
// expanded into tile T0).  Returns the output descriptor (DESC_EMPTY for an
// empty result or a failed allocation).
__device__ __noinline__ uint64_t warp_probe_pair(ExecState *es, WChunk &wc, uint32_t op, const CRef &a,
                                                 const CRef &b, uint64_t *T0, uint64_t *T1, uint32_t lane) {
    const bool a_arr = a.type == T_ARRAY, b_arr = b.type == T_ARRAY;
    const CRef *X, *O;
    uint32_t want = 1;
    if (op == OP_AND) {
        if (a_arr && b_arr) X = a.card <= b.card ? &a : &b;
        else X = a_arr ? &a : &b;
        O = (X == &a) ? &b : &a;
    } else {
        X = &a;
        O = &b;
        want = 0;
    }
    const uint64_t *ow;
    if (O->type == T_BITSET) {
        ow = reinterpret_cast<const uint64_t *>(O->p);
    } else {
        t_decode(T0, *O, lane);
        ow = T0;
    }
    uint16_t *L = reinterpret_cast<uint16_t *>(T1);
    const uint32_t c = probe_list<true>(reinterpret_cast<const uint16_t *>(X->p), X->card, ow, want, L, lane);
    if (c == 0) return DESC_EMPTY;
    const uint32_t r = list_runs(L, c, lane);
    const uint32_t ty = canon_type(c, r);
    const uint64_t off = chunk_alloc_words(es, wc, word_alloc_bytes(ty, c, r), lane);
    if (off == ALLOC_FAIL) return DESC_EMPTY;
    if (ty == T_ARRAY) l_emit_array(L, c, reinterpret_cast<uint16_t *>(es->arena + off), lane);
    else l_emit_runs(L, c, r, reinterpret_cast<uint16_t *>(T0), reinterpret_cast<uint32_t *>(es->arena + off), lane);
    return mk_desc(c, ty, ty == T_RUN ? r : 0, off);
}

// |a n b| for one container pair with an array operand: bit tests of the
// smaller array's values against the other container
__device__ __noinline__ uint32_t warp_probe_count(const CRef &a, const CRef &b, uint64_t *T0, uint32_t lane) {
    const bool a_arr = a.type == T_ARRAY, b_arr = b.type == T_ARRAY;
    const CRef *X = (a_arr && b_arr) ? (a.card <= b.card ? &a : &b) : (a_arr ? &a : &b);
    const CRef *O = (X == &a) ? &b : &a;
    const uint64_t *ow;
    if (O->type == T_BITSET) ow = reinterpret_cast<const uint64_t *>(O->p);
    else { t_decode(T0, *O, lane); ow = T0; }
    const uint32_t c = probe_list<false>(reinterpret_cast<const uint16_t *>(X->p), X->card, ow, 1, nullptr, lane);
    __syncwarp();
    return c;
}

// ------------------------------------------------------------ key merge

// number of a's keys among the first d elements of the merge of a and b
// (a first on a tie), by a cooperative 32-ary search: each round the warp
// evaluates "a[i] precedes b[d-1-i]" at 32 evenly spaced i and keeps the
// stretch where it turns false (4 rounds for 65536 keys)
__device__ __forceinline__ uint32_t merge_split(const uint16_t *ka, uint32_t na, const uint16_t *kb, uint32_t nb,
                                                uint32_t d, uint32_t lane) {
    uint32_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
#pragma unroll 1
    while (hi > lo) {
        const uint32_t span = hi - lo;
        if (span <= 32) {
            bool pr = false;
            if (lane < span) {
                const uint32_t i = lo + lane;
                pr = __ldg(ka + i) <= __ldg(kb + (d - 1 - i));
            }
            lo += __popc(__ballot_sync(FULL, pr));
            break;
        }
        const uint32_t step = (span + 31) / 32;
        const uint32_t i = lo + lane * step;
        bool pr = false;
        if (i < hi) pr = __ldg(ka + i) <= __ldg(kb + (d - 1 - i));
        const uint32_t k = __popc(__ballot_sync(FULL, pr));
        if (k == 0) break;   // a[lo] does not precede: the split is lo
        const uint32_t nlo = lo + (k - 1) * step + 1;
        hi = min(hi, lo + k * step);
        lo = nlo;
    }
    return lo;
}

// ------------------------------------------------------------ array merges

// Sec. 1 membership rule as a 4-bit table indexed by (element comes from a) * 2
// + (the other input has it): AND keeps a's shared values, OR keeps all of a
// and b's unshared ones, ANDNOT a's unshared ones, XOR every unshared value
__device__ __forceinline__ uint32_t keep_table(uint32_t op) {
    return op == OP_AND ? 0x8u : op == OP_OR ? 0xDu : op == OP_ANDNOT ? 0x4u : 0x5u;
}

// one lane merges two small sorted arrays without branches on the data: each
// step compares the two heads, keeps the smaller one (either one when they
// are equal, and then both advance) by the op's table, and advances the
// input(s) it came from; counts cardinality c and runs r, and with EMIT
// writes the kept values to out (4-byte aligned; whole words are written,
// the upper half of an odd last word zeroed).  a and b are generic pointers:
// the arrays staged in shared memory, or in global memory.  TBL is the op's
// table (keep_table), fixed at compile time so that each op's loop carries
// only its own keep test.
template <bool EMIT, uint32_t TBL>
__device__ __forceinline__ void lane_merge_arrays_t(const uint16_t *a, uint32_t na, const uint16_t *b, uint32_t nb,
                                                    uint32_t &c, uint32_t &r, uint16_t *out) {
    // what the table keeps: a value only a holds (bit 2), only b holds
    // (bit 0), both hold (bit 3, taken from a)
    constexpr bool k_a = (TBL & 4u) != 0, k_b = (TBL & 1u) != 0, k_ab = (TBL & 8u) != 0;
    uint32_t i = 0, j = 0, last = 0xFFFFFFFEu;
    c = 0;
    r = 0;
    // once one input is exhausted the rest of the other is kept whole or
    // dropped whole: AND stops at the first end, ANDNOT once a ends, OR and
    // XOR run to both ends
#pragma unroll 1
    while ((i < na && (j < nb || k_a)) || (j < nb && k_b)) {
        const uint32_t va = i < na ? (uint32_t)a[i] : KEY_END;
        const uint32_t vb = j < nb ? (uint32_t)b[j] : KEY_END;
        const bool lt = va < vb, gt = vb < va;
        const uint32_t v = gt ? vb : va;
        if (lt ? k_a : gt ? k_b : k_ab) {
            // kept values leave in pairs, one 4-byte store per two values
            if (EMIT && (c & 1u)) reinterpret_cast<uint32_t *>(out)[c >> 1] = last | (v << 16);
            r += (v != last + 1);
            last = v;
            c++;
        }
        i += !gt;
        j += !lt;
    }
    if (EMIT && (c & 1u)) reinterpret_cast<uint32_t *>(out)[c >> 1] = last;   // zero upper half
}

// the merge above for a table known only at run time
template <bool EMIT>
__device__ __forceinline__ void lane_merge_arrays(uint32_t tbl, const uint16_t *a, uint32_t na, const uint16_t *b,
                                                  uint32_t nb, uint32_t &c, uint32_t &r, uint16_t *out) {
    switch (tbl) {
        case 0x8u: lane_merge_arrays_t<EMIT, 0x8u>(a, na, b, nb, c, r, out); break;
        case 0xDu: lane_merge_arrays_t<EMIT, 0xDu>(a, na, b, nb, c, r, out); break;
        case 0x4u: lane_merge_arrays_t<EMIT, 0x4u>(a, na, b, nb, c, r, out); break;
        default: lane_merge_arrays_t<EMIT, 0x5u>(a, na, b, nb, c, r, out); break;
    }
}

// |a n b| of two small sorted arrays by one lane: equal heads count and both
// advance, otherwise the smaller head advances
__device__ __forceinline__ uint32_t lane_count_and(const uint16_t *a, uint32_t na, const uint16_t *b, uint32_t nb) {
    uint32_t i = 0, j = 0, c = 0;
#pragma unroll 1
    while (i < na && j < nb) {
        const uint32_t va = a[i], vb = b[j];
        c += va == vb;
        i += va <= vb;
        j += vb <= va;
    }
    return c;
}

// ------------------------------------------------------------ lean kernel

// hint the first `lines` 128-byte lines of a payload into L2
__device__ __forceinline__ void prefetch_payload(const uint8_t *p, uint32_t bytes, uint32_t lines) {
    const uint32_t n = min((bytes + 127) / 128, lines);
    for (uint32_t i = 0; i < n; i++) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 128 * i));
}

enum : uint32_t { M_NONE = 0, M_LANE_ARR, M_LANE_SWEEP, M_COPY, M_WARP_ARR, M_DEFER, M_GRP_ARR };
constexpr uint32_t WARP_MERGE_MAX = 1024;   // values of both arrays the warp merges through shared memory
// array pairs merged GPER at a time by groups of GW lanes, each group staging
// in a GSEG-element region (at most GRP_MAX values, so that whole words fit)
constexpr uint32_t GW = 8, GSEG = 256, GPER = 32 / GW;
constexpr uint32_t GRP_MAX = GSEG - 2;
constexpr uint32_t RUN_SWEEP_MAX = 512;     // intervals one lane sweeps when runs are involved
constexpr uint32_t LSTG_WORDS = WARP_MERGE_MAX;   // 4-byte words of the staging area (4 KB)

// bytes reserved for an array-by-array result before it is computed: the
// array encoding of the largest possible result (the run encoding, chosen
// only when smaller, also fits)
__device__ __forceinline__ uint32_t array_result_bound(uint32_t op, uint32_t na, uint32_t nb) {
    const uint32_t n = op == OP_AND ? min(na, nb) : op == OP_ANDNOT ? na : na + nb;
    return (2 * n + 3) & ~3u;
}

// The array and run containers that a tile's lanes copy unchanged (mine), by
// the whole warp: one allocation in lane order, so the destination is one
// contiguous stretch; the source is one stretch too when every copied
// container follows the previous one (consecutive keys of one input), and
// otherwise each destination word finds its container by a search over the
// lanes' word offsets.  The words move 128 per round, 4 loads per lane in
// flight; the first round is read before the allocation returns.  Writes
// the results and adds them to the query's sums.
__device__ __forceinline__ void copy_tile(ExecState *es, unsigned long long *wa, unsigned long long pos_base, bool mine,
                                       uint64_t dx, const uint8_t *base, uint32_t key, uint32_t pos,
                                       unsigned long long &acc, uint32_t lane) {
    const uint32_t ty = d_type(dx), c = d_card(dx), r = ty == T_RUN ? d_runs(dx) : 0;
    const uint32_t bytes = mine ? word_alloc_bytes(ty, c, r) : 0;
    const uint32_t incl = warp_incl(bytes, lane), total = __shfl_sync(FULL, incl, 31);
    const uint32_t nw = bytes / 4, wincl = incl / 4, T = total / 4;
    const unsigned long long src = mine ? (unsigned long long)(base + d_off(dx)) : 0ull;
    const uint32_t cm = __ballot_sync(FULL, mine);
    const uint32_t below = cm & lanemask_lt(lane);
    const int prev = below ? 31 - __clz(below) : (int)lane;
    const unsigned long long pend = __shfl_sync(FULL, src + 4ull * nw, prev);
    const bool one = __all_sync(FULL, !mine || !below || src == pend);
    const uint32_t *S1 = reinterpret_cast<const uint32_t *>(__shfl_sync(FULL, src, __ffs(cm) - 1));
    // word g of the tile's copies: its container is the lane j whose words
    // [wincl_j - nw_j, wincl_j) hold g, found by a 5-step search over lanes
    auto gather = [&](uint32_t g) -> uint32_t {
        uint32_t j = 0;
#pragma unroll
        for (uint32_t s = 16; s; s >>= 1)
            if (__shfl_sync(FULL, wincl, j + s - 1) <= g) j += s;
        const uint32_t *S = reinterpret_cast<const uint32_t *>(__shfl_sync(FULL, src, j));
        const uint32_t ex = __shfl_sync(FULL, wincl - nw, j);
        return g < T ? __ldg(S + (g - ex)) : 0u;
    };
    // The first round is read before the allocation returns.  A contiguous
    // source is copied to a destination placed at the same address modulo
    // 16 (the allocation takes 12 bytes more), so that its 16-byte-aligned
    // body moves as 16-byte vectors, 512 words per round (4 per lane in
    // flight), and at most 3 words at each end move alone; a gathered source
    // moves 128 words per round (4 loads, each after its container search).
    unsigned long long wbase = 0;
    uint32_t shift = 0;
    bool ok = true;
    uint32_t *D = nullptr;
    if (one) {
        const uint64_t s0 = reinterpret_cast<uint64_t>(S1);
        const uint32_t hw = min((uint32_t)(((16u - (uint32_t)(s0 & 15u)) & 15u) >> 2), T);   // head words
        const uint32_t nv = (T - hw) >> 2, tw = T - hw - 4 * nv;                            // body vectors, tail words
        const uint4 *SV = reinterpret_cast<const uint4 *>(S1 + hw);
        const bool has_h = lane < hw, has_t = lane >= 4 && lane < 4 + tw;
        const uint32_t hv = has_h ? __ldg(S1 + lane) : 0u;
        const uint32_t tv = has_t ? __ldg(S1 + hw + 4 * nv + (lane - 4)) : 0u;
        for (uint32_t v0 = 0;; v0 += 32 * 4) {
            uint4 x[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t vi = v0 + 32u * k + lane;
                x[k] = vi < nv ? __ldg(SV + vi) : make_uint4(0u, 0u, 0u, 0u);
            }
            if (v0 == 0) {
                wbase = lean_alloc(es, wa, total + 12, lane);
                ok = wbase != ALLOC_FAIL;
                if (!ok) break;
                const uint64_t d0 = reinterpret_cast<uint64_t>(es->arena + es->words_off + wbase);
                shift = (uint32_t)((s0 - d0) & 15u);
                D = reinterpret_cast<uint32_t *>(d0 + shift);
                if (has_h) D[lane] = hv;
                if (has_t) D[hw + 4 * nv + (lane - 4)] = tv;
            }
            uint4 *DV = reinterpret_cast<uint4 *>(D + hw);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const uint32_t vi = v0 + 32u * k + lane;
                if (vi < nv) DV[vi] = x[k];
            }
            if (v0 + 32 * 4 >= nv) break;
        }
    } else
    for (uint32_t g0 = 0;; g0 += 128) {
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) v[k] = g0 + 32u * k < T ? gather(g0 + 32u * k + lane) : 0u;
        if (g0 == 0) {
            wbase = lean_alloc(es, wa, total, lane);
            ok = wbase != ALLOC_FAIL;
            if (!ok) break;
            D = reinterpret_cast<uint32_t *>(es->arena + es->words_off + wbase);
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (g0 + 32u * k + lane < T) D[g0 + 32u * k + lane] = v[k];
        if (g0 + 128 >= T) break;
    }
    if (mine) {
        es->descs[pos_base + pos] = ok ? mk_desc(c, ty, r, es->words_off + wbase + shift + incl - bytes) : DESC_EMPTY;
        es->keys[pos_base + pos] = (uint16_t)key;
        acc += in_payload_bytes(dx) + (ok ? payload_bytes(ty, c, r) + META_BYTES : 0);
    }
    // the query's sums gather in the warp's shared state (wa[2], wa[3]) and
    // are flushed when the warp leaves the query
    const uint32_t csum = warp_sum(mine ? c : 0);
    if (lane == 0 && ok) {
        wa[2] += csum;
        wa[3] += total;
    }
}

// add the sums a warp gathered for query p to its stats
__device__ __forceinline__ void flush_sums(PairStats *stats, uint32_t p, unsigned long long *wa, uint32_t lane) {
    if (lane == 0) {
        if (wa[2]) atomicAdd(&stats[p].card, wa[2]);
        if (wa[3]) atomicAdd(&stats[p].words, wa[3]);
        wa[2] = wa[3] = 0;
    }
    __syncwarp();
}

// driver mode (skewed AND/ANDNOT/count queries), out of the hot path: slot's
// key from the driving list, found in the other by binary search; returns
// kind | key << 16, ia, ib
__device__ __noinline__ uint4 resolve_driven(const BmView &A, const BmView &B, uint32_t slot, bool and_like,
                                             bool count_only) {
    uint32_t kind, key, ia = 0, ib = 0;
    if (and_like) {
        const bool drvA = A.n <= B.n;
        const uint16_t *dk = drvA ? A.keys : B.keys;
        const uint16_t *ok = drvA ? B.keys : A.keys;
        const uint32_t on = drvA ? B.n : A.n;
        key = __ldg(dk + slot);
        const uint32_t j = lower_bound16(ok, on, key);
        if (j < on && __ldg(ok + j) == key) {
            kind = K_PAIR;
            ia = drvA ? slot : j;
            ib = drvA ? j : slot;
        } else {
            kind = count_only ? K_NONE : K_EMPTY;
        }
    } else {   // ANDNOT, driven by a
        key = __ldg(A.keys + slot);
        const uint32_t j = lower_bound16(B.keys, B.n, key);
        ia = slot;
        if (j < B.n && __ldg(B.keys + j) == key) {
            kind = K_PAIR;
            ib = j;
        } else {
            kind = K_COPY_A;
        }
    }
    return make_uint4(kind | (key << 16), ia, ib, 0u);
}

// append the tile's container pairs for the heavy kernel (lanes in lm)
__device__ __noinline__ void queue_deferred(ExecState *es, uint32_t lm, bool mine, uint64_t da, uint64_t db, uint32_t p,
                                            uint32_t pos, uint32_t kind_key, uint32_t lane) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&es->defer_n, (unsigned long long)__popc(lm));
    base = __shfl_sync(FULL, base, 0);
    if (mine) {
        const unsigned long long at = base + __popc(lm & lanemask_lt(lane));
        if (at < es->defer_cap) {
            Deferred d;
            d.da = da;
            d.db = db;
            d.p = p;
            d.pos = pos;
            d.kind_key = kind_key;
            d.pad = 0;
            es->defer[at] = d;
        } else {
            atomicOr(&es->status, 2u);
        }
    }
}

// Small-pair queue slots are taken SQCHUNK at a time from the shared
// counters; each warp hands out its current block ([qs[0], qs[1]) for
// one-lane items, [qs[2], qs[3]) for the others) and moves to a new block in
// the middle of a tile when one runs out, so that the only unused slots are
// the rest of each warp's last blocks, which k_lean fills with no-op items
// before it ends.
constexpr uint32_t SQCHUNK = 256;
__device__ __forceinline__ unsigned long long sq_take(unsigned long long *ctr, unsigned long long *qs, uint32_t cnt,
                                                      uint32_t k, uint32_t lane) {
    const unsigned long long cur = qs[0], end = qs[1], rem = end - cur;
    unsigned long long nb = 0;
    if (cnt > rem) {
        if (lane == 0) nb = atomicAdd(ctr, (unsigned long long)SQCHUNK);
        nb = __shfl_sync(FULL, nb, 0);
    }
    __syncwarp();
    if (lane == 0) {
        if (cnt > rem) {
            qs[0] = nb + (cnt - rem);
            qs[1] = nb + SQCHUNK;
        } else {
            qs[0] = cur + cnt;
        }
    }
    __syncwarp();
    return k < rem ? cur + k : nb + (k - rem);
}

// append the tile's small container pairs (lanes in am) to the small-pair
// queue: one-lane items (one1) from the bottom, the others from the top
__device__ __forceinline__ void queue_small(ExecState *es, unsigned long long *qs, uint32_t am, bool mine, bool one1,
                                         uint64_t da, uint64_t db, uint32_t p, uint32_t pos, uint32_t info,
                                         uint32_t lane) {
    const uint32_t m1 = __ballot_sync(FULL, mine && one1), m2 = am & ~m1;
    unsigned long long k1 = 0, k2 = 0;
    if (m1) k1 = sq_take(&es->small_n1, qs, __popc(m1), __popc(m1 & lanemask_lt(lane)), lane);
    if (m2) k2 = sq_take(&es->small_n2, qs + 2, __popc(m2), __popc(m2 & lanemask_lt(lane)), lane);
    if (mine) {
        const unsigned long long k = one1 ? k1 : k2;
        if (k < es->small_cap) {
            Item it;
            it.da = da;
            it.db = db;
            it.p = p;
            it.pos = pos;
            it.info = info;
            it.pad = 0;
            es->small[one1 ? k : es->small_cap - 1 - k] = it;
        } else {
            atomicOr(&es->status, 2u);
        }
    }
}

// no-op items in the unused rest of a warp's blocks (mode M_NONE)
__device__ __noinline__ void sq_close(ExecState *es, const unsigned long long *qs, uint32_t lane) {
    for (int c = 0; c < 2; c++) {
        for (unsigned long long k = qs[2 * c] + lane; k < qs[2 * c + 1]; k += 32) {
            if (k >= es->small_cap) break;
            Item it;
            it.da = it.db = 0;
            it.p = it.pos = it.info = it.pad = 0;
            es->small[c == 0 ? k : es->small_cap - 1 - k] = it;
        }
    }
}

// Key merge of one tile: each lane resolves its slot into a container pair,
// an empty result, a copy or nothing.  Empty results and copies of array and
// run containers are finished at once, pairs with a bitset or many values go
// to the heavy kernel's queue, and the others to the small-pair queue.
//
// Tiles come in chunks of consecutive ones, and the cursor carries what the
// previous tile found: its query's tile range, so that the query is looked up
// again only when the tile leaves it, and where its merge ended, so that the
// merge-path search runs only for a chunk's first tile.
struct TileCursor {
    unsigned long long lo, hi;   // tiles of query p
    unsigned long long t_next;   // tile whose merge starts at a's key i_next
    uint32_t p, i_next;
};

__device__ void resolve_tile(const PairParams &P, unsigned long long t, TileCursor &cur, uint32_t *win,
                             unsigned long long *wa, unsigned long long &meta, uint32_t lane) {
    if (t < cur.lo || t >= cur.hi) {
        flush_sums(P.stats, cur.p, wa, lane);
        uint32_t lo = 0, hi = P.n_pairs;
#pragma unroll 1
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (P.tile_base[mid] <= t) lo = mid;
            else hi = mid;
        }
        cur.p = lo;
        cur.lo = P.tile_base[lo];
        cur.hi = lo + 1 < P.n_pairs ? P.tile_base[lo + 1] : P.n_tiles;
    }
    const uint32_t p = cur.p;
    const PairDev pd = P.pairs[p];
    const BmView A = P.qv[p].a, B = P.qv[p].b;
    ExecState *es = P.es;
    const uint32_t op = pd.op;
    const bool count_only = (pd.flags & F_COUNT) != 0;
    const uint32_t local = (uint32_t)(t - cur.lo);

    uint32_t kind = K_NONE, key = 0, pos = 0, ia = 0, ib = 0;
    if (pd.flags & F_MERGE) {
        const uint32_t d0 = local * 32u;
        const uint32_t i0 = local == 0         ? 0u
                            : t == cur.t_next ? cur.i_next
                                              : merge_split(A.keys, A.n, B.keys, B.n, d0, lane);
        const uint32_t j0 = d0 - i0;
        uint32_t *WA = win;        // WA[0] = a[i0-1], WA[1..32] = a[i0..i0+31]
        uint32_t *WB = win + 33;   // WB[0..31] = b[j0..j0+31]
        WA[1 + lane] = i0 + lane < A.n ? (uint32_t)__ldg(A.keys + i0 + lane) : KEY_END;
        WB[lane] = j0 + lane < B.n ? (uint32_t)__ldg(B.keys + j0 + lane) : KEY_END;
        if (lane == 0) WA[0] = i0 > 0 ? (uint32_t)__ldg(A.keys + i0 - 1) : 0xFFFFFFFFu;
        __syncwarp();
        uint32_t a_upto = 0;   // a's keys among this tile's first lane + 1 elements
        if (d0 + lane < A.n + B.n) {
            // x = a's keys among this tile's first `lane` elements
            uint32_t xl = 0, xh = lane;
#pragma unroll 1
            while (xl < xh) {
                const uint32_t m = (xl + xh) >> 1;
                if (WA[1 + m] <= WB[lane - 1 - m]) xl = m + 1;
                else xh = m;
            }
            const uint32_t av = WA[1 + xl], bv = WB[lane - xl];
            const uint32_t ai = i0 + xl, bj = j0 + lane - xl;
            a_upto = xl + (av <= bv);
            if (av <= bv) {   // a's key ai; b has it too iff bv == av
                key = av;
                const bool m = bv == av;
                pos = (op == OP_OR || op == OP_XOR) ? d0 + lane : ai;
                ia = ai;
                ib = bj;
                if (count_only) kind = m ? K_PAIR : K_NONE;
                else if (m) kind = K_PAIR;
                else kind = (op == OP_AND) ? K_EMPTY : K_COPY_A;
            } else {          // b's key bj; shared iff a's previous key equals it
                key = bv;
                const bool m = WA[xl] == bv;
                if (!count_only && (op == OP_OR || op == OP_XOR)) {
                    pos = d0 + lane;
                    ib = bj;
                    kind = m ? K_EMPTY : K_COPY_B;
                }
            }
        }
        cur.t_next = t + 1;
        cur.i_next = i0 + __shfl_sync(FULL, a_upto, 31);
        __syncwarp();
    } else {
        const uint32_t slot = local * 32u + lane;
        if (slot < pd.n_slots) {
            const uint4 rs = resolve_driven(A, B, slot, count_only || op == OP_AND, count_only);
            kind = rs.x & 0xFFFFu;
            key = rs.x >> 16;
            pos = slot;
            ia = rs.y;
            ib = rs.z;
        }
    }
    const uint64_t da = (kind == K_PAIR || kind == K_COPY_A) ? __ldg(A.descs + ia) : 0ull;
    const uint64_t db = (kind == K_PAIR || kind == K_COPY_B) ? __ldg(B.descs + ib) : 0ull;

    // who does the work: one lane (array merges, run sweeps), the whole warp
    // (copies, large array pairs) or the heavy kernel
    uint32_t mode = M_NONE;
    if (kind == K_PAIR) {
        const uint32_t ta = d_type(da), tb = d_type(db);
        if (ta == T_ARRAY && tb == T_ARRAY) {
            const uint32_t n = d_card(da) + d_card(db);
            mode = n <= P.small_iv ? M_LANE_ARR
                   : n <= GRP_MAX        ? M_GRP_ARR
                   : n <= WARP_MERGE_MAX - 2 ? M_WARP_ARR
                                             : M_DEFER;
        } else if (ta != T_BITSET && tb != T_BITSET && n_intervals(da) + n_intervals(db) <= RUN_SWEEP_MAX) {
            mode = M_LANE_SWEEP;
        } else {
            mode = M_DEFER;
        }
    } else if (kind == K_COPY_A || kind == K_COPY_B) {
        const uint64_t dx = kind == K_COPY_A ? da : db;
        mode = d_type(dx) == T_BITSET ? M_DEFER : M_COPY;
    }
    const uint32_t lm = __ballot_sync(FULL, mode == M_DEFER);
    if (lm) queue_deferred(es, lm, mode == M_DEFER, da, db, p, pos, (kind << 16) | key, lane);
    if (kind == K_EMPTY) {
        es->descs[pd.pos_base + pos] = DESC_EMPTY;
        es->keys[pd.pos_base + pos] = (uint16_t)key;
    }
    if (__any_sync(FULL, mode == M_COPY))
        copy_tile(es, wa, pd.pos_base, mode == M_COPY, kind == K_COPY_B ? db : da,
                  kind == K_COPY_B ? B.base : A.base, key, pos, meta, lane);
    const bool act = mode != M_NONE && mode != M_DEFER && mode != M_COPY;
    if (act && P.prefetch) {
        // start fetching the payloads into L2 now; the queue is processed
        // after one or two more tiles have been resolved
        prefetch_payload(A.base + d_off(da), in_payload_bytes(da), P.prefetch);
        prefetch_payload(B.base + d_off(db), in_payload_bytes(db), P.prefetch);
    }
    const uint32_t am = __ballot_sync(FULL, act);
    if (am) queue_small(es, wa + 4, am, act, mode == M_LANE_ARR || mode == M_LANE_SWEEP, da, db, p, pos,
                        key | (kind << 16) | (mode << 20), lane);
}

// The first 32 four-byte words of both arrays of a warp-sized pair, one per
// lane, loaded ahead: the warp requests the next pair's while it merges the
// current one.  Array payloads start 4-byte aligned and are padded to 4 bytes.
struct WPre {
    uint32_t a, b;
};
__device__ __forceinline__ WPre prefetch_words(const uint16_t *ga, uint32_t na, const uint16_t *gb, uint32_t nb,
                                               uint32_t lane) {
    WPre w;
    w.a = lane < (na + 1) / 2 ? __ldg(reinterpret_cast<const uint32_t *>(ga) + lane) : 0u;
    w.b = lane < (nb + 1) / 2 ? __ldg(reinterpret_cast<const uint32_t *>(gb) + lane) : 0u;
    return w;
}

// a then b in shared memory as whole words (b starts at element 2 * ceil(na / 2);
// na + nb <= 1022 fits 1024 elements), from the prefetched words and the rest
// of the arrays; returns b's start
__device__ __forceinline__ uint16_t *stage_words(const uint16_t *ga, uint32_t na, const uint16_t *gb, uint32_t nb,
                                                 const WPre &w, uint16_t *stg, uint32_t lane) {
    const uint32_t wa = (na + 1) / 2, wb = (nb + 1) / 2;
    uint32_t *SA = reinterpret_cast<uint32_t *>(stg), *SB = SA + wa;
    if (lane < wa) SA[lane] = w.a;
    if (lane < wb) SB[lane] = w.b;
#pragma unroll 1
    for (uint32_t x = 32 + lane; x < wa; x += 32) SA[x] = __ldg(reinterpret_cast<const uint32_t *>(ga) + x);
#pragma unroll 1
    for (uint32_t x = 32 + lane; x < wb; x += 32) SB[x] = __ldg(reinterpret_cast<const uint32_t *>(gb) + x);
    __syncwarp();
    return stg + 2 * wa;
}

// |a n b| of two sorted arrays (na + nb <= 1022) by the warp, for the
// count-only forms: staged as below, each lane walks its merge-path chunk
// and counts the values of a that b holds too
__device__ __noinline__ uint32_t warp_count_arrays(const uint16_t *ga, uint32_t na, const uint16_t *gb, uint32_t nb,
                                                   const WPre &w, uint16_t *stg, uint32_t lane) {
    const uint16_t *SA = stg, *SB = stage_words(ga, na, gb, nb, w, stg, lane);
    const uint32_t tot = na + nb, L = (tot + 31) >> 5;
    const uint32_t d = min(lane * L, tot), dend = min(d + L, tot);
    uint32_t lo = d > nb ? d - nb : 0, hi = min(d, na);
#pragma unroll 1
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (SA[m] <= SB[d - 1 - m]) lo = m + 1;
        else hi = m;
    }
    uint32_t i = lo, j = d - lo, c = 0;
#pragma unroll 1
    for (uint32_t s = d; s < dend; s++) {
        const uint32_t va = i < na ? (uint32_t)SA[i] : KEY_END, vb = j < nb ? (uint32_t)SB[j] : KEY_END;
        const bool ta = va <= vb;
        c += ta && va == vb;
        i += ta;
        j += !ta;
    }
    const uint32_t C = warp_sum(c);
    __syncwarp();
    return C;
}

// The warp merges two sorted arrays (na + nb <= 1022) through shared memory:
// coalesced staging, the merged sequence cut into 32 equal chunks found by
// merge-path binary search, one chunk per lane (recording which input each
// step took and which values it kept), a warp scan to place the kept values,
// and the canonical encoding.  off is the reserved output (ALLOC_FAIL: count
// only).  Returns the descriptor; card gets the cardinality.
__device__ __noinline__ uint64_t warp_merge_arrays(ExecState *es, uint32_t tbl, const uint16_t *ga, uint32_t na,
                                                   const uint16_t *gb, uint32_t nb, const WPre &w, uint16_t *stg,
                                                   uint32_t lane, uint64_t off, uint32_t &card) {
    uint16_t *SA = stg, *SB = stage_words(ga, na, gb, nb, w, stg, lane), *SO = stg + WARP_MERGE_MAX;
    const uint32_t tot = na + nb, L = (tot + 31) >> 5;
    const uint32_t d = min(lane * L, tot), dend = min(d + L, tot);
    uint32_t lo = d > nb ? d - nb : 0, hi = min(d, na);
#pragma unroll 1
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (SA[m] <= SB[d - 1 - m]) lo = m + 1;
        else hi = m;
    }
    const uint32_t i0 = lo, j0 = d - lo;
    uint32_t i = i0, j = j0, pa = i0 > 0 ? (uint32_t)SA[i0 - 1] : 0xFFFFFFFFu;
    uint32_t take_a = 0, kept = 0, c = 0, r = 0, first = 0, last = 0xFFFFFFFEu;
#pragma unroll 1
    for (uint32_t s = 0; d + s < dend; s++) {
        const uint32_t va = i < na ? (uint32_t)SA[i] : KEY_END, vb = j < nb ? (uint32_t)SB[j] : KEY_END;
        const bool ta = va <= vb;
        const uint32_t v = ta ? va : vb;
        const bool ino = ta ? (vb == va) : (pa == vb);
        take_a |= (uint32_t)ta << s;
        if ((tbl >> ((ta ? 2u : 0u) | (ino ? 1u : 0u))) & 1u) {
            kept |= 1u << s;
            if (c == 0) first = v;
            r += (v != last + 1);
            last = v;
            c++;
        }
        pa = ta ? va : pa;
        i += ta;
        j += !ta;
    }
    // a lane's first kept value continues a run when it follows the last kept
    // value of the lanes before it (values increase, so a max-scan finds it)
    uint32_t m = c ? last + 1 : 0;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, m, dd);
        if (lane >= (uint32_t)dd) m = max(m, y);
    }
    uint32_t prev = __shfl_up_sync(FULL, m, 1);
    if (lane == 0) prev = 0;
    if (c && prev != 0 && first == prev) r--;
    const uint32_t cincl = warp_incl(c, lane);
    const uint32_t C = __shfl_sync(FULL, cincl, 31), R = warp_sum(r);
    card = C;
    uint64_t desc = DESC_EMPTY;
    if (off != ALLOC_FAIL && C) {
        const uint32_t ty = canon_type(C, R);   // C <= 1024: array or runs
        uint32_t qq = cincl - c;
        i = i0;
        j = j0;
#pragma unroll 1
        for (uint32_t s = 0; d + s < dend; s++) {
            const bool ta = (take_a >> s) & 1u;
            const uint16_t v = ta ? SA[i] : SB[j];
            i += ta;
            j += !ta;
            if ((kept >> s) & 1u) SO[qq++] = v;
        }
        __syncwarp();
        if (ty == T_ARRAY) l_emit_array(SO, C, reinterpret_cast<uint16_t *>(es->arena + off), lane);
        else l_emit_runs(SO, C, R, stg, reinterpret_cast<uint32_t *>(es->arena + off), lane);
        desc = mk_desc(C, ty, ty == T_RUN ? R : 0, off);
    }
    __syncwarp();
    return desc;
}

// ------------------------------------------------------------ group merges
// Array pairs of at most GRP_MAX values are merged four at a time, each by a
// group of GW = 8 lanes, with the same steps as the warp merge above (staged
// inputs, merge-path chunks, scans over the group, canonical encoding).  A
// group's staging region is GSEG elements of the warp's first half of stg,
// its output region the same stretch of the second half.  Every lane of the
// warp runs these functions (idle groups with na = nb = 0); the shuffles sit
// outside the loops whose trip counts differ between groups.

__device__ __forceinline__ uint32_t g_incl(uint32_t x, uint32_t sl) {
#pragma unroll
    for (uint32_t d = 1; d < GW; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, d, GW);
        if (sl >= d) x += y;
    }
    return x;
}
__device__ __forceinline__ uint32_t g_sum(uint32_t x) {
#pragma unroll
    for (uint32_t d = GW / 2; d; d >>= 1) x += __shfl_xor_sync(FULL, x, d, GW);
    return x;
}

// both arrays of a group's pair, a then b as whole words (b starts at element
// 2 * ceil(na / 2)); 16 loads per lane in flight, the rest (more than 128
// words, na + nb > 254) by a second loop
__device__ __forceinline__ uint16_t *g_stage(const uint16_t *ga, uint32_t na, const uint16_t *gb, uint32_t nb,
                                             uint16_t *S, uint32_t sl) {
    const uint32_t wa = (na + 1) / 2, wt = wa + (nb + 1) / 2;
    const uint32_t *A32 = reinterpret_cast<const uint32_t *>(ga), *B32 = reinterpret_cast<const uint32_t *>(gb);
    uint32_t *S32 = reinterpret_cast<uint32_t *>(S);
    uint32_t v[16];
#pragma unroll
    for (uint32_t k = 0; k < 16; k++) {
        const uint32_t x = k * GW + sl;
        v[k] = x < wt ? __ldg(x < wa ? A32 + x : B32 + (x - wa)) : 0u;
    }
#pragma unroll
    for (uint32_t k = 0; k < 16; k++) {
        const uint32_t x = k * GW + sl;
        if (x < wt) S32[x] = v[k];
    }
#pragma unroll 1
    for (uint32_t x = 16 * GW + sl; x < wt; x += GW) S32[x] = __ldg(x < wa ? A32 + x : B32 + (x - wa));
    __syncwarp();
    return S + 2 * wa;
}

// the merge-path split of a group lane's chunk: its first element d, its end,
// and how many of a's values precede d
struct GChunk {
    uint32_t d, dend, i0;
};
__device__ __forceinline__ GChunk g_chunk(const uint16_t *SA, uint32_t na, const uint16_t *SB, uint32_t nb,
                                          uint32_t sl) {
    const uint32_t tot = na + nb, L = (tot + GW - 1) / GW;
    GChunk g;
    g.d = min(sl * L, tot);
    g.dend = min(g.d + L, tot);
    uint32_t lo = g.d > nb ? g.d - nb : 0, hi = min(g.d, na);
#pragma unroll 1
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (SA[m] <= SB[g.d - 1 - m]) lo = m + 1;
        else hi = m;
    }
    g.i0 = lo;
    return g;
}

// a op b for a group's pair (na + nb <= GRP_MAX) into the reserved output
// off (ALLOC_FAIL: nothing written); returns the descriptor on every lane of
// the group, card gets the cardinality
__device__ __noinline__ uint64_t group_merge_arrays(ExecState *es, uint32_t tbl, const uint16_t *ga, uint32_t na,
                                                    const uint16_t *gb, uint32_t nb, uint16_t *SI, uint16_t *SO,
                                                    uint32_t sl, uint64_t off, uint32_t &card) {
    const uint16_t *SA = SI, *SB = g_stage(ga, na, gb, nb, SI, sl);
    const GChunk g = g_chunk(SA, na, SB, nb, sl);
    uint32_t i = g.i0, j = g.d - g.i0, pa = g.i0 > 0 ? (uint32_t)SA[g.i0 - 1] : 0xFFFFFFFFu;
    uint32_t take_a = 0, kept = 0, c = 0, r = 0, first = 0, last = 0xFFFFFFFEu;
#pragma unroll 1
    for (uint32_t s = 0; g.d + s < g.dend; s++) {
        const uint32_t va = i < na ? (uint32_t)SA[i] : KEY_END, vb = j < nb ? (uint32_t)SB[j] : KEY_END;
        const bool ta = va <= vb;
        const uint32_t v = ta ? va : vb;
        const bool ino = ta ? (vb == va) : (pa == vb);
        take_a |= (uint32_t)ta << s;
        if ((tbl >> ((ta ? 2u : 0u) | (ino ? 1u : 0u))) & 1u) {
            kept |= 1u << s;
            if (c == 0) first = v;
            r += (v != last + 1);
            last = v;
            c++;
        }
        pa = ta ? va : pa;
        i += ta;
        j += !ta;
    }
    // a lane's first kept value continues a run when it follows the last kept
    // value of the group's lanes before it (a max-scan finds that value)
    uint32_t m = c ? last + 1 : 0;
#pragma unroll
    for (uint32_t dd = 1; dd < GW; dd <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, m, dd, GW);
        if (sl >= dd) m = max(m, y);
    }
    uint32_t prev = __shfl_up_sync(FULL, m, 1, GW);
    if (sl == 0) prev = 0;
    if (c && prev != 0 && first == prev) r--;
    const uint32_t cincl = g_incl(c, sl), rincl = g_incl(r, sl);
    const uint32_t C = __shfl_sync(FULL, cincl, GW - 1, GW), R = __shfl_sync(FULL, rincl, GW - 1, GW);
    card = C;
    const bool emit = off != ALLOC_FAIL && C != 0;
    const uint32_t ty = canon_type(C, R);   // C <= GRP_MAX: array or runs
    if (emit) {
        uint32_t qq = cincl - c;
        i = g.i0;
        j = g.d - g.i0;
#pragma unroll 1
        for (uint32_t s = 0; g.d + s < g.dend; s++) {
            const bool ta = (take_a >> s) & 1u;
            const uint16_t v = ta ? SA[i] : SB[j];
            i += ta;
            j += !ta;
            if ((kept >> s) & 1u) SO[qq++] = v;
        }
    }
    __syncwarp();
    if (emit && ty == T_RUN) {
        // run starts of this lane's kept values, indexed by run, into the
        // (no longer needed) staging region
        uint32_t q0 = cincl - c, k = rincl - r;
#pragma unroll 1
        for (uint32_t x = q0; x < q0 + c; x++)
            if (x == 0 || (uint32_t)SO[x] != (uint32_t)SO[x - 1] + 1) SI[k++] = (uint16_t)x;
    }
    __syncwarp();
    uint64_t desc = DESC_EMPTY;
    if (emit) {
        if (ty == T_ARRAY) {
            uint16_t *out = reinterpret_cast<uint16_t *>(es->arena + off);
#pragma unroll 1
            for (uint32_t x = sl; x < C; x += GW) out[x] = SO[x];
        } else {
            uint32_t *out = reinterpret_cast<uint32_t *>(es->arena + off);
#pragma unroll 1
            for (uint32_t x = sl; x < R; x += GW) {
                const uint32_t s = SI[x], e = (x + 1 < R ? (uint32_t)SI[x + 1] : C) - 1;
                out[x] = (uint32_t)SO[s] | ((uint32_t)(SO[e] - SO[s]) << 16);
            }
        }
        desc = mk_desc(C, ty, ty == T_RUN ? R : 0, off);
    }
    __syncwarp();
    return desc;
}

// |a n b| for a group's pair (na + nb <= GRP_MAX), on every lane of the group
__device__ __noinline__ uint32_t group_count_arrays(const uint16_t *ga, uint32_t na, const uint16_t *gb, uint32_t nb,
                                                    uint16_t *SI, uint32_t sl) {
    const uint16_t *SA = SI, *SB = g_stage(ga, na, gb, nb, SI, sl);
    const GChunk g = g_chunk(SA, na, SB, nb, sl);
    uint32_t i = g.i0, j = g.d - g.i0, c = 0;
#pragma unroll 1
    for (uint32_t s = g.d; s < g.dend; s++) {
        const uint32_t va = i < na ? (uint32_t)SA[i] : KEY_END, vb = j < nb ? (uint32_t)SB[j] : KEY_END;
        const bool ta = va <= vb;
        c += ta && va == vb;
        i += ta;
        j += !ta;
    }
    const uint32_t C = g_sum(c);
    __syncwarp();
    return C;
}

// Group-sized array merges of the lanes in gq, GPER at a time: group g of
// lanes takes the g-th of the next GPER queued pairs; each served lane gets
// its pair's descriptor and cardinality
__device__ __forceinline__ void process_groups(ExecState *es, uint32_t gq, const CRef &ca, const CRef &cb, uint32_t tbl,
                                            uint64_t off, bool count, uint16_t *stg, uint32_t lane, uint64_t &desc,
                                            uint32_t &card) {
    const uint32_t g = lane / GW, sl = lane % GW;
    uint16_t *GI = stg + GSEG * g, *GO = stg + WARP_MERGE_MAX + GSEG * g;
#pragma unroll 1
    while (gq) {
        // the (up to) GPER queued lanes served now; group g takes the
        // g-th of them
        uint32_t rest = gq;
#pragma unroll
        for (uint32_t x = 0; x < GPER; x++) rest &= rest - 1;
        const uint32_t taken = gq & ~rest;
        gq = rest;
        uint32_t mine_g = taken;
        for (uint32_t x = 0; x < g; x++) mine_g &= mine_g - 1;
        const uint32_t src = mine_g ? (uint32_t)__ffs(mine_g) - 1 : 32u;
        const uint32_t s = src < 32 ? src : 0;
        const unsigned long long pa_s = __shfl_sync(FULL, (unsigned long long)ca.p, s);
        const unsigned long long pb_s = __shfl_sync(FULL, (unsigned long long)cb.p, s);
        uint32_t na_s = __shfl_sync(FULL, ca.card, s), nb_s = __shfl_sync(FULL, cb.card, s);
        const uint32_t tbl_s = __shfl_sync(FULL, tbl, s);
        const uint64_t off_s = __shfl_sync(FULL, count ? ALLOC_FAIL : off, s);
        const bool cnt_s = __shfl_sync(FULL, (uint32_t)count, s) != 0;
        if (src == 32) na_s = nb_s = 0;
        uint32_t c = 0;
        uint64_t dsc = DESC_EMPTY;
        // count-only and materialising queries may share a batch: both
        // functions run on every lane, each group uses its own result
        const bool any_cnt = __any_sync(FULL, src < 32 && cnt_s);
        const bool any_mat = __any_sync(FULL, src < 32 && !cnt_s);
        if (any_cnt) {
            const uint32_t cc = group_count_arrays(reinterpret_cast<const uint16_t *>(pa_s), cnt_s ? na_s : 0,
                                                   reinterpret_cast<const uint16_t *>(pb_s), cnt_s ? nb_s : 0, GI,
                                                   sl);
            if (cnt_s) c = cc;
        }
        if (any_mat) {
            uint32_t cm = 0;
            const uint64_t dm = group_merge_arrays(es, tbl_s, reinterpret_cast<const uint16_t *>(pa_s),
                                                   cnt_s ? 0 : na_s, reinterpret_cast<const uint16_t *>(pb_s),
                                                   cnt_s ? 0 : nb_s, GI, GO, sl, off_s, cm);
            if (!cnt_s) {
                c = cm;
                dsc = dm;
            }
        }
        // each served lane reads its group's result from the group's first lane
        const uint32_t mine = (taken >> lane) & 1u ? __popc(taken & lanemask_lt(lane)) : 0u;
        const uint32_t c_r = __shfl_sync(FULL, c, mine * GW);
        const uint64_t d_r = __shfl_sync(FULL, dsc, mine * GW);
        if ((taken >> lane) & 1u) {
            desc = d_r;
            card = c_r;
        }
    }
}

// Warp-sized array merges of the lanes in wq, one at a time; the first words
// of the next pair are requested before the current one is merged; each
// served lane gets its pair's descriptor and cardinality
__device__ __noinline__ void process_warp_merges(ExecState *es, uint32_t wq, const CRef &ca, const CRef &cb,
                                                 uint32_t tbl, uint64_t off, bool count, uint16_t *stg, uint32_t lane,
                                                 uint64_t &desc, uint32_t &card) {
    auto pre = [&](int k) -> WPre {
        return prefetch_words(reinterpret_cast<const uint16_t *>(__shfl_sync(FULL, (unsigned long long)ca.p, k)),
                              __shfl_sync(FULL, ca.card, k),
                              reinterpret_cast<const uint16_t *>(__shfl_sync(FULL, (unsigned long long)cb.p, k)),
                              __shfl_sync(FULL, cb.card, k), lane);
    };
    WPre w_cur = {0u, 0u};
    if (wq) w_cur = pre(__ffs(wq) - 1);
    while (wq) {
        const int src = __ffs(wq) - 1;
        wq &= wq - 1;
        WPre w_next = {0u, 0u};
        if (wq) w_next = pre(__ffs(wq) - 1);
        const uint32_t tbl_s = __shfl_sync(FULL, tbl, src);
        const uint64_t off_s = __shfl_sync(FULL, count ? ALLOC_FAIL : off, src);
        const unsigned long long pa_s = __shfl_sync(FULL, (unsigned long long)ca.p, src);
        const unsigned long long pb_s = __shfl_sync(FULL, (unsigned long long)cb.p, src);
        const uint32_t na_s = __shfl_sync(FULL, ca.card, src), nb_s = __shfl_sync(FULL, cb.card, src);
        uint32_t c = 0;
        uint64_t dsc = DESC_EMPTY;
        if (__shfl_sync(FULL, (uint32_t)count, src))
            c = warp_count_arrays(reinterpret_cast<const uint16_t *>(pa_s), na_s,
                                  reinterpret_cast<const uint16_t *>(pb_s), nb_s, w_cur, stg, lane);
        else
            dsc = warp_merge_arrays(es, tbl_s, reinterpret_cast<const uint16_t *>(pa_s), na_s,
                                    reinterpret_cast<const uint16_t *>(pb_s), nb_s, w_cur, stg, lane, off_s, c);
        w_cur = w_next;
        if (lane == (uint32_t)src) {
            desc = dsc;
            card = c;
        }
    }
}

// Process n <= 32 queued container pairs q[0, n), one per lane (group- and
// warp-sized ones by 8 lanes or the whole warp in turn), with one allocation
// for all their outputs.  The queue holds pairs only: copies are done during
// the key merge.  stg is the warp's 4 KB staging area.
__device__ void process_items(const PairParams &P, const Item *q, uint32_t n, uint16_t *stg, unsigned long long *wa,
                              unsigned long long &bytes_acc, uint32_t lane) {
    ExecState *es = P.es;
    Item it;
    it.da = it.db = 0;
    it.p = it.pos = it.info = it.pad = 0;
    if (lane < n) it = q[lane];
    const bool has = lane < n && ((it.info >> 20) & 7u) != M_NONE;   // no-op items fill unused queue slots
    const uint32_t mode = has ? (it.info >> 20) & 7u : M_NONE;
    const uint32_t key = it.info & 0xFFFFu;
    const PairDev pd = P.pairs[it.p];
    const uint8_t *abase = P.qv[it.p].a.base, *bbase = P.qv[it.p].b.base;
    const bool count = (pd.flags & F_COUNT) != 0;
    const uint32_t op = count ? (uint32_t)OP_AND : pd.op;
    const uint32_t tbl = keep_table(op);
    const CRef ca = cref(abase, it.da), cb = cref(bbase, it.db);

    // One-lane array merges read both arrays from the warp's staging area:
    // every lane's words are requested at once (cp.async), so the warp waits
    // for one memory latency, not once for every cache line a lane reaches
    // (the lines of 32 lanes' arrays do not stay in L1 at this occupancy).
    // Lanes whose words would pass the end of the area read global memory.
    const uint16_t *la = reinterpret_cast<const uint16_t *>(ca.p), *lb = reinterpret_cast<const uint16_t *>(cb.p);
    if (__any_sync(FULL, mode == M_LANE_ARR)) {
        const uint32_t wa = mode == M_LANE_ARR ? (ca.card + 1) / 2 : 0, wb = mode == M_LANE_ARR ? (cb.card + 1) / 2 : 0;
        const uint32_t wincl = warp_incl(wa + wb, lane);
        if (mode == M_LANE_ARR && wincl <= LSTG_WORDS) {
            uint32_t *S = reinterpret_cast<uint32_t *>(stg) + (wincl - wa - wb);
            const uint32_t *A32 = reinterpret_cast<const uint32_t *>(ca.p), *B32 = reinterpret_cast<const uint32_t *>(cb.p);
#pragma unroll 1
            for (uint32_t k = 0; k < wa; k++) cp_async4(S + k, A32 + k);
#pragma unroll 1
            for (uint32_t k = 0; k < wb; k++) cp_async4(S + wa + k, B32 + k);
            la = reinterpret_cast<const uint16_t *>(S);
            lb = reinterpret_cast<const uint16_t *>(S + wa);
        }
        cp_async_wait_all();
        __syncwarp();
    }

    // sizes: exact for run sweeps, the array bound for array merges
    uint32_t bytes = 0, lc = 0, lr = 0, lt = 0;
    if (!count) {
        if (mode == M_LANE_ARR || mode == M_WARP_ARR || mode == M_GRP_ARR) {
            bytes = array_result_bound(op, ca.card, cb.card);
        } else if (mode == M_LANE_SWEEP) {
            lane_sweep<false>(op, iv_src(ca), iv_src(cb), lc, lr, 0, nullptr);
            if (lc) {
                lt = canon_type(lc, lr);
                bytes = word_alloc_bytes(lt, lc, lr);
            }
        }
    }
    // one allocation for the batch
    const uint32_t incl = warp_incl(bytes, lane), total = __shfl_sync(FULL, incl, 31);
    unsigned long long wbase = 0;
    bool ok = true;
    if (total) {
        wbase = lean_alloc(es, wa, total, lane);
        ok = wbase != ALLOC_FAIL;
    }
    const uint64_t off = (ok && bytes) ? es->words_off + wbase + incl - bytes : ALLOC_FAIL;

    uint64_t desc = DESC_EMPTY;
    uint32_t card = 0;
    if (mode == M_LANE_ARR) {
        uint32_t c, r;
        if (count) {
            c = lane_count_and(la, ca.card, lb, cb.card);
            r = 0;
        } else if (off == ALLOC_FAIL) {
            lane_merge_arrays<false>(tbl, la, ca.card, lb, cb.card, c, r, nullptr);
        } else {
            lane_merge_arrays<true>(tbl, la, ca.card, lb, cb.card, c, r, reinterpret_cast<uint16_t *>(es->arena + off));
            if (c) {
                const uint32_t ty = canon_type(c, r);
                if (ty == T_RUN) {   // rare: rewrite the reserved space as runs
                    uint32_t c2, r2;
                    lane_sweep<true>(op, iv_src(ca), iv_src(cb), c2, r2, T_RUN, es->arena + off);
                }
                desc = mk_desc(c, ty, ty == T_RUN ? r : 0, off);
            }
        }
        card = c;
    } else if (mode == M_LANE_SWEEP) {
        if (count) {
            uint32_t r;
            lane_sweep<false>(op, iv_src(ca), iv_src(cb), card, r, 0, nullptr);
        } else if (lc && off != ALLOC_FAIL) {
            uint32_t c2, r2;
            lane_sweep<true>(op, iv_src(ca), iv_src(cb), c2, r2, lt, es->arena + off);
            desc = mk_desc(lc, lt, lt == T_RUN ? lr : 0, off);
            card = lc;
        }
    }
    __syncwarp();   // the staging area is free again
    // group-sized array merges, GPER at a time
    const uint32_t gq = __ballot_sync(FULL, mode == M_GRP_ARR);
    if (gq) process_groups(es, gq, ca, cb, tbl, off, count, stg, lane, desc, card);
    // warp-sized array merges, one at a time (pairs of 255..1022 values)
    const uint32_t wq = __ballot_sync(FULL, mode == M_WARP_ARR);
    if (wq) process_warp_merges(es, wq, ca, cb, tbl, off, count, stg, lane, desc, card);
    // results, and per-query sums over the lanes of the same query
    if (has && !count) {
        es->descs[pd.pos_base + it.pos] = desc;
        es->keys[pd.pos_base + it.pos] = (uint16_t)key;
    }
    const uint32_t words = (desc != DESC_EMPTY) ? word_alloc_bytes(d_type(desc), d_card(desc), d_runs(desc)) : 0;
    const uint32_t grp = __match_any_sync(FULL, has ? it.p : 0xFFFFFFFFu);
    const uint32_t csum = __reduce_add_sync(grp, card), wsum = __reduce_add_sync(grp, words);
    if (has && lane == (uint32_t)(__ffs(grp) - 1)) {
        if (csum) atomicAdd(&P.stats[it.p].card, (unsigned long long)csum);
        if (wsum) atomicAdd(&P.stats[it.p].words, (unsigned long long)wsum);
    }
    if (has) {
        bytes_acc += in_payload_bytes(it.da) + in_payload_bytes(it.db);
        if (desc != DESC_EMPTY) bytes_acc += payload_bytes(d_type(desc), d_card(desc), d_runs(desc)) + META_BYTES;
    }
}

__global__ void __launch_bounds__(LEAN_THREADS, LEAN_CTAS_MAX) k_lean(PairParams P) {
    __shared__ uint32_t s_win[LEAN_THREADS / 32][66];
    // per warp: word-region chunk and query sums (0..3), small-queue blocks (4..7)
    __shared__ unsigned long long s_alloc[LEAN_THREADS / 32][8];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < 8) s_alloc[warp][lane] = 0;
    __syncwarp();
    unsigned long long bytes_acc = 0, t = 0, t_end = 0;
    TileCursor cur;
    cur.lo = cur.hi = 0;
    cur.t_next = ~0ull;
    cur.p = cur.i_next = 0;
    for (;;) {
        if (t == t_end) {
            if (lane == 0) t = atomicAdd(&P.es->work, (unsigned long long)P.chunk);
            t = __shfl_sync(FULL, t, 0);
            if (t >= P.n_tiles) break;
            t_end = min(t + P.chunk, P.n_tiles);
        }
        resolve_tile(P, t, cur, s_win[warp], s_alloc[warp], bytes_acc, lane);
        t++;
    }
    sq_close(P.es, s_alloc[warp] + 4, lane);
    flush_sums(P.stats, cur.p, s_alloc[warp], lane);
    const unsigned long long tot = warp_sum64(bytes_acc);
    if (lane == 0 && tot) atomicAdd(&P.es->lean_bytes, tot);
}

// ------------------------------------------------------------ small-pair kernel

// The small container pairs k_lean queued, by a persistent kernel whose warps
// take 32 queued pairs at a time: first every one-lane item (array merges of
// at most small_iv values, run sweeps), then the group and warp items (array
// pairs merged by 8 lanes, four at once, or by the whole warp).  All warps
// work through one phase before the next, so each phase's code stays hot.
constexpr uint32_t SMALL_CTAS_MAX = 8;
__global__ void __launch_bounds__(LEAN_THREADS, SMALL_CTAS_MAX) k_small(PairParams P) {
    __shared__ __align__(16) uint16_t s_stg[LEAN_THREADS / 32][2 * WARP_MERGE_MAX];
    __shared__ unsigned long long s_alloc[LEAN_THREADS / 32][4];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ExecState *es = P.es;
    if (lane == 0) s_alloc[warp][0] = s_alloc[warp][1] = s_alloc[warp][2] = s_alloc[warp][3] = 0;
    __syncwarp();
    const unsigned long long cap = es->small_cap, n1 = es->small_n1, n2 = es->small_n2;
    if (n1 + n2 > cap) return;   // the queue overflowed: the host reruns with exact sizes
    unsigned long long bytes_acc = 0;
    bool second = false;   // phase: one-lane items, then group and warp items
    for (;;) {
        const unsigned long long n = second ? n2 : n1;
        unsigned long long x = 0;
        if (lane == 0) x = atomicAdd(second ? &es->swork2 : &es->swork1, 32ull);
        x = __shfl_sync(FULL, x, 0);
        if (x >= n) {
            if (second) break;
            second = true;
            continue;
        }
        process_items(P, es->small + (second ? cap - n2 : 0ull) + x, (uint32_t)min(32ull, n - x), s_stg[warp],
                      s_alloc[warp], bytes_acc, lane);
    }
    const unsigned long long tot = warp_sum64(bytes_acc);
    if (lane == 0 && tot) atomicAdd(&es->small_bytes, tot);
}

// ------------------------------------------------------------ heavy kernel

// bulk-copy state of one heavy-kernel warp, and the warp's current chunk of
// the bitset region ([bcur, bend), taken HCHUNK bitsets at a time)
struct Tma {
    uint64_t *bar;
    uint32_t phase;
    bool failed;
    unsigned long long bcur, bend;
    WChunk wc;   // the warp's chunk of the word region
};
constexpr uint32_t HCHUNK = 8;

// one 8 KB slot of the bitset region for the warp: from its chunk, or a new
// chunk from the shared counter (at most HCHUNK - 1 slots per warp go unused;
// the arena adds that slack)
__device__ __forceinline__ uint64_t heavy_alloc_bitset(ExecState *es, Tma &t, uint32_t lane) {
    if (t.bcur + 8192ull > t.bend) {
        unsigned long long old = 0;
        if (lane == 0) old = atomicAdd(&es->bits_used, 8192ull * HCHUNK);
        old = __shfl_sync(FULL, old, 0);
        if (old + 8192ull * HCHUNK > es->bits_cap) {
            if (lane == 0) atomicOr(&es->status, 1u);
            t.bcur = t.bend = 0;
            return ALLOC_FAIL;
        }
        t.bcur = old;
        t.bend = old + 8192ull * HCHUNK;
    }
    const uint64_t off = es->bits_off + t.bcur;
    t.bcur += 8192ull;
    return off;
}

// a wait ran out: record it, give the copy in flight one more bounded wait,
// and stop using the tiles
__device__ bool tma_fail(Tma &t, ExecState *es, uint32_t lane) {
    if (lane == 0) atomicOr(&es->status, 4u);
    mbar_wait(t.bar, t.phase ^ 1u);
    t.failed = true;
    return false;
}

// Stage both operands of a pair in the warp's tiles: bitsets arrive by bulk
// copy (a -> T0, b -> T1) while the warp expands array and run operands into
// the other tile.  False if a wait ran out.
__device__ __noinline__ bool stage_pair(const CRef &a, const CRef &b, uint64_t *T0, uint64_t *T1, Tma &t, ExecState *es,
                           uint32_t lane) {
    const uint32_t nbits = (a.type == T_BITSET) + (b.type == T_BITSET);
    if (nbits) {
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
            mbar_expect_tx(t.bar, nbits * 8192u);
            if (a.type == T_BITSET) bulk_load(T0, a.p, 8192u, t.bar);
            if (b.type == T_BITSET) bulk_load(T1, b.p, 8192u, t.bar);
        }
    }
    if (a.type != T_BITSET) t_decode(T0, a, lane);
    if (b.type != T_BITSET) t_decode(T1, b, lane);
    if (nbits) {
        const bool ok = mbar_wait(t.bar, t.phase);
        t.phase ^= 1u;
        if (!ok) return tma_fail(t, es, lane);
    }
    return true;
}

// write tile T0 as a bitset container with one bulk store
__device__ __noinline__ uint64_t store_bitset_tile(ExecState *es, Tma &t, const uint64_t *T0, uint32_t c,
                                                   uint32_t lane) {
    const uint64_t off = heavy_alloc_bitset(es, t, lane);
    if (off == ALLOC_FAIL) return DESC_EMPTY;
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
        bulk_store(es->arena + off, T0, 8192u);
        bulk_wait_read();
    }
    __syncwarp();
    return mk_desc(c, T_BITSET, 0, off);
}

// a op b for one deferred container pair
__device__ __noinline__ uint64_t heavy_pair(ExecState *es, uint32_t op, const CRef &a, const CRef &b, uint64_t *T0, uint64_t *T1,
                               Tma &t, uint32_t lane) {
    const bool a_arr = a.type == T_ARRAY, b_arr = b.type == T_ARRAY;
    if ((op == OP_AND && (a_arr || b_arr)) || (op == OP_ANDNOT && a_arr))
        return warp_probe_pair(es, t.wc, op, a, b, T0, T1, lane);
    if (!stage_pair(a, b, T0, T1, t, es, lane)) return DESC_EMPTY;
    uint32_t c, r;
    t_combine<true>(T0, T0, T1, op, c, r, lane);
    __syncwarp();
    if (c == 0) return DESC_EMPTY;
    const uint32_t ty = canon_type(c, r);
    if (ty == T_BITSET) return store_bitset_tile(es, t, T0, c, lane);
    const uint64_t off = chunk_alloc_words(es, t.wc, word_alloc_bytes(ty, c, r), lane);
    if (off == ALLOC_FAIL) return DESC_EMPTY;
    if (ty == T_ARRAY) {
        t_emit_array(T0, reinterpret_cast<uint16_t *>(es->arena + off), lane);
    } else {
        uint16_t *S = reinterpret_cast<uint16_t *>(T1);
        t_emit_runs(T0, S, S + 2048, reinterpret_cast<uint32_t *>(es->arena + off), r, lane);
    }
    __syncwarp();
    return mk_desc(c, ty, ty == T_RUN ? r : 0, off);
}

// copy of a deferred container: bitsets through shared memory by bulk copy
__device__ __noinline__ uint64_t heavy_copy(ExecState *es, const CRef &x, uint64_t *T0, uint64_t *T1, Tma &t, uint32_t lane) {
    if (x.type != T_BITSET) return warp_copy(es, x, lane);
    (void)T1;
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
        mbar_expect_tx(t.bar, 8192u);
        bulk_load(T0, x.p, 8192u, t.bar);
    }
    const bool ok = mbar_wait(t.bar, t.phase);
    t.phase ^= 1u;
    if (!ok) {
        tma_fail(t, es, lane);
        return DESC_EMPTY;
    }
    return store_bitset_tile(es, t, T0, x.card, lane);
}

// |a n b| for one deferred container pair
__device__ __noinline__ uint32_t heavy_count(const CRef &a, const CRef &b, uint64_t *T0, uint64_t *T1, Tma &t, ExecState *es,
                                uint32_t lane) {
    if (a.type == T_ARRAY || b.type == T_ARRAY) return warp_probe_count(a, b, T0, lane);
    if (!stage_pair(a, b, T0, T1, t, es, lane)) return 0;
    uint32_t c, r;
    t_combine<false>(nullptr, T0, T1, OP_AND, c, r, lane);
    __syncwarp();
    return c;
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) k_heavy(PairParams P) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ __align__(8) uint64_t s_bar[WARPS];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *T0 = smem + (size_t)warp * 2048;
    uint64_t *T1 = T0 + 1024;
    ExecState *es = P.es;
    if (lane == 0) mbar_init(&s_bar[warp], 1);
    fence_mbar_init();
    __syncwarp();
    Tma t;
    t.bar = &s_bar[warp];
    t.phase = 0;
    t.failed = false;
    t.bcur = t.bend = 0;
    t.wc.cur = t.wc.end = 0;
    unsigned long long hbytes = 0;   // algorithmic bytes of this warp's items (lane 0)
    const unsigned long long n = min(es->defer_n, es->defer_cap);
    // the next item's index and record are fetched while this one is worked on
    auto next = [&](Deferred &d) -> unsigned long long {
        unsigned long long x = 0;
        if (lane == 0) x = atomicAdd(&es->hwork, 1ull);
        x = __shfl_sync(FULL, x, 0);
        if (x < n) d = es->defer[x];
        return x;
    };
    Deferred Dn;
    unsigned long long en = next(Dn);
    for (;;) {
        if (en >= n || t.failed) break;
        const Deferred D = Dn;
        en = next(Dn);
        const PairDev pd = P.pairs[D.p];
        const BmView A = P.qv[D.p].a, B = P.qv[D.p].b;
        const uint32_t kind = D.kind_key >> 16, key = D.kind_key & 0xFFFFu;
        PairStats *S = P.stats + D.p;
        if (pd.flags & F_COUNT) {
            const uint32_t c = heavy_count(cref(A.base, D.da), cref(B.base, D.db), T0, T1, t, es, lane);
            if (lane == 0) {
                if (c) atomicAdd(&S->card, (unsigned long long)c);
                hbytes += in_payload_bytes(D.da) + in_payload_bytes(D.db);
            }
            __syncwarp();
            continue;
        }
        uint64_t desc;
        unsigned long long ib;
        if (kind == K_PAIR) {
            desc = heavy_pair(es, pd.op, cref(A.base, D.da), cref(B.base, D.db), T0, T1, t, lane);
            ib = in_payload_bytes(D.da) + in_payload_bytes(D.db);
        } else {
            const uint64_t dx = kind == K_COPY_A ? D.da : D.db;
            desc = heavy_copy(es, cref(kind == K_COPY_A ? A.base : B.base, dx), T0, T1, t, lane);
            ib = in_payload_bytes(dx);
        }
        if (lane == 0) {
            es->descs[pd.pos_base + D.pos] = desc;
            es->keys[pd.pos_base + D.pos] = (uint16_t)key;
            if (desc != DESC_EMPTY) {
                const uint32_t ty = d_type(desc), c = d_card(desc), r = d_runs(desc);
                atomicAdd(&S->card, (unsigned long long)c);
                if (ty == T_BITSET) atomicAdd(&S->nbits, 1u);
                else atomicAdd(&S->words, (unsigned long long)word_alloc_bytes(ty, c, r));
                ib += payload_bytes(ty, c, r) + META_BYTES;
            }
            hbytes += ib;
        }
        __syncwarp();
    }
    if (lane == 0 && hbytes) atomicAdd(&es->heavy_bytes, hbytes);
    // every bulk store of this warp has completed before the kernel ends
    if (lane == 0) bulk_wait_all();
    __syncwarp();
}

// drop empty results: in-place stream compaction of each query's output
// range (positions are already in key order), one block per query
// blocks take queries from a shared counter in the order `order` gives
// (materialising queries by decreasing number of positions, so that the
// largest are not left for the end)
__global__ void __launch_bounds__(512) k_compact(const PairDev *pairs, const uint32_t *order, uint32_t n_order,
                                                 PairStats *stats, ExecState *es) {
    __shared__ uint32_t s_w[16];
    __shared__ uint32_t s_tot, s_next;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (;;) {
        if (tid == 0) s_next = (uint32_t)atomicAdd(&es->cwork, 1ull);
        __syncthreads();
        const uint32_t x = s_next;
        __syncthreads();
        if (x >= n_order) break;
        const uint32_t p = order[x];
        const PairDev pd = pairs[p];
        const uint32_t n = pd.n_pos;
        uint64_t *D = es->descs + pd.pos_base;
        uint16_t *K = es->keys + pd.pos_base;
        uint32_t out = 0;
        for (uint32_t c0 = 0; c0 < n; c0 += blockDim.x) {
            const uint32_t i = c0 + tid;
            const uint64_t d = i < n ? D[i] : DESC_EMPTY;
            const uint16_t k = i < n ? K[i] : 0;
            const uint32_t f = d != DESC_EMPTY;
            const uint32_t m = __ballot_sync(FULL, f);
            if (lane == 0) s_w[warp] = __popc(m);
            __syncthreads();
            if (warp == 0) {
                const uint32_t v = lane < nw ? s_w[lane] : 0;
                const uint32_t inc = warp_incl(v, lane);
                if (lane < nw) s_w[lane] = inc - v;
                if (lane == 31) s_tot = inc;
            }
            __syncthreads();
            if (f) {
                const uint32_t q = out + s_w[warp] + __popc(m & lanemask_lt(lane));
                D[q] = d;
                K[q] = k;
            }
            out += s_tot;
            __syncthreads();
        }
        if (tid == 0) stats[p].n_out = out;
    }
}

// ------------------------------------------------------------ host side

// k_heavy's dynamic shared-memory limits, raised once per device (function
// attributes belong to the current device's context)
void init_kernel_attrs() {
    constexpr int MAX_DEV = 256;
    static std::atomic<int> done[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return;
    if (dev < MAX_DEV && done[dev].load(std::memory_order_relaxed)) return;
    cudaFuncSetAttribute(k_heavy<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 16384);
    cudaFuncSetAttribute(k_heavy<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 16384);
    cudaFuncSetAttribute(k_heavy<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 16384);
    if (dev < MAX_DEV) done[dev].store(1, std::memory_order_relaxed);
}

template <int W>
void launch_heavy_w(const PairParams &P, int ctas_per_sm, cudaStream_t s) {
    const unsigned grid = (unsigned)std::max(1, sm_count() * ctas_per_sm);
    k_heavy<W><<<grid, W * 32, W * 16384, s>>>(P);
}

}  // namespace

#include <thread>

struct rb_plan {
    std::vector<const rb *> pool;
    std::vector<rb_query> q;
    std::vector<PairDev> pairs;
    uint64_t total_pos = 0, total_tiles = 0;
    uint64_t words_cap = 0, bits_cap = 0, defer_cap = 0;   // arena sizes for the next run
    uint64_t small_cap = 0;                                // small-pair queue entries for the next run
    bool exact = false;                                    // caps measured by a previous run
    bool any_mat = false;
    uint8_t *tables = nullptr;
    uint64_t tables_bytes = 0;
    BmView *d_pool = nullptr;
    PairDev *d_pairs = nullptr;
    QViews *d_qv = nullptr;
    unsigned long long *d_tile_base = nullptr;
    PairStats *d_stats = nullptr;
    ExecState *d_es = nullptr;
    uint32_t *d_order = nullptr;   // materialising queries by decreasing positions (k_compact)
    uint32_t n_order = 0;
    PairStats *h_stats = nullptr;
    ExecState *h_es = nullptr;
    cudaStream_t ps = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr, ev_in = nullptr, ev_done = nullptr;
    RbArena *pending = nullptr;   // result memory of a run launched by rb_plan_launch, not yet collected
    bool pending_graph = false;
    cudaStream_t pending_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    rb_schedule gsched = {0, 0, 0, 0, 0, 0};
    double last_ms = 0, last_lean_ms = 0, last_small_ms = 0, last_heavy_ms = 0;
    uint64_t last_alg = 0, last_out = 0, last_lean_bytes = 0, last_small_bytes = 0, last_heavy_bytes = 0;
    uint64_t last_deferred = 0, last_small = 0;
    uint64_t meta_bytes = 0;   // algorithmic key + metadata bytes of the inputs (and count results)
    cudaStream_t alloc_stream = nullptr;
};

namespace {

void plan_destroy(rb_plan *p) {
    if (!p) return;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->tables) dev_free(p->tables, p->tables_bytes, p->alloc_stream);
    if (p->h_stats) cudaFreeHost(p->h_stats);
    if (p->h_es) cudaFreeHost(p->h_es);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->ev2) cudaEventDestroy(p->ev2);
    if (p->ev3) cudaEventDestroy(p->ev3);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    if (p->pending) {
        if (p->ps) cudaStreamSynchronize(p->ps);
        arena_unref(p->pending);
    }
    if (p->ps) cudaStreamDestroy(p->ps);
    delete p;
}

// per-query bound on output bytes, used when a run has no measured sizes:
// a canonical result container is never larger than twice the payload of
// its inputs (its run or array encoding), and a bitset output needs more
// than 4096 values
void query_bounds(const rb *A, const rb *B, uint32_t op, uint64_t &w, uint64_t &bits) {
    const uint64_t pa = A->word_bytes + 8192ull * A->n_bitsets, pb = B->word_bytes + 8192ull * B->n_bitsets;
    const uint64_t slots = op == OP_AND ? std::min(A->n, B->n) : op == OP_ANDNOT ? A->n : (uint64_t)A->n + B->n;
    const uint64_t cards = op == OP_AND ? std::min(A->card, B->card) : op == OP_ANDNOT ? A->card : A->card + B->card;
    uint64_t wb;
    if (op == OP_AND) wb = 2 * std::min(pa, pb);
    else if (op == OP_ANDNOT) wb = 2 * pa;
    else wb = 2 * (pa + pb);
    w = wb + 4 * slots;
    bits = 8192ull * std::min<uint64_t>(slots, cards / 4097 + 1);
}

uint64_t lean_warps(const rb_plan *p, const rb_schedule &sc);

// Host passes over a batch's queries run in up to 8 pieces of at least
// 8,192 queries on their own threads (the caller takes the first piece):
// building a 65,536-query plan is otherwise a few milliseconds of one core.
uint32_t plan_pieces(uint64_t n) {
    if (n < 2 * 8192) return 1;
    static const uint64_t hw = std::max(1u, std::thread::hardware_concurrency());   // read once
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(std::min<uint64_t>(hw, 8), n / 8192));
}
template <class F>
void parallel_pieces(uint64_t n, uint32_t pieces, F f) {
    const uint64_t per = (n + pieces - 1) / std::max<uint32_t>(pieces, 1);
    std::vector<std::thread> th;
    for (uint32_t k = 1; k < pieces; k++) {
        const uint64_t lo = k * per, hi = std::min(n, lo + per);
        if (lo >= hi) continue;
        try {
            th.emplace_back(f, k, lo, hi);
        } catch (...) {   // no thread to be had: the caller runs the piece
            f(k, lo, hi);
        }
    }
    f(0u, (uint64_t)0, std::min(n, per));
    for (std::thread &t : th) t.join();
}

rb_status plan_build(const rb_t *const *pool, uint32_t pool_n, const rb_query *q, uint64_t nq, cudaStream_t s,
                     bool use_bounds, rb_plan **out) {
    *out = nullptr;
    if (nq && (!pool || !q)) return set_err(RB_EINVAL, "batch: NULL pool or queries");
    if (nq > 0xFFFFFFFFull) return set_err(RB_ERANGE, "batch: too many queries");
    for (uint32_t i = 0; i < pool_n; i++)
        if (!pool[i]) return set_err(RB_EINVAL, "batch: pool[%u] is NULL", i);
    rb_plan *p = new rb_plan;
    p->alloc_stream = s;
    p->pool.assign(pool, pool + pool_n);
    p->q.assign(q, q + nq);
    p->pairs.resize(nq);
    std::vector<unsigned long long> tb(nq + 1);
    for (uint64_t i = 0; i < nq; i++) {
        const rb_query &x = q[i];
        if (x.op > 3 || x.a >= pool_n || x.b >= pool_n) {
            plan_destroy(p);
            return set_err(RB_EINVAL, "batch: query %llu has op %u, a %u, b %u (pool of %u)",
                           (unsigned long long)i, x.op, x.a, x.b, pool_n);
        }
    }
    // per query: its mode, slots and positions, and its share of the size
    // estimates (in parallel pieces; the offsets are summed up after)
    struct Sums {
        uint64_t meta = 0, small_bound = 0, ed = 0, ew = 0, eb = 0, bw = 0, bb = 0;
        bool any_mat = false;
    };
    const uint32_t pieces = plan_pieces(nq);
    std::vector<Sums> part(pieces);
    parallel_pieces(nq, pieces, [&](uint32_t k, uint64_t lo, uint64_t hi) {
        Sums &S = part[k];
        for (uint64_t i = lo; i < hi; i++) {
            const rb_query &x = q[i];
            const rb *A = pool[x.a], *B = pool[x.b];
            PairDev &d = p->pairs[i];
            d.a = x.a;
            d.b = x.b;
            d.op = x.op;
            const bool count = (x.flags & RB_Q_COUNT_ONLY) != 0;
            const uint64_t na = A->n, nb = B->n, mn = std::min(na, nb), mx = std::max(na, nb);
            // merge mode unless one key list is more than 8 times the other
            // (then a binary search per key of the smaller side is cheaper)
            bool merge;
            if (!count && (x.op == OP_OR || x.op == OP_XOR)) merge = true;
            else if (!count && x.op == OP_ANDNOT) merge = !(nb * 8 < na || na * 8 < nb);
            else merge = mx <= 8 * mn;
            d.flags = (count ? F_COUNT : 0) | (merge ? F_MERGE : 0);
            // the key arrays and metadata of both inputs, and a count-only result
            S.meta += META_BYTES * (na + nb) + (count ? COUNT_BYTES : 0);
            uint64_t ns, np;
            if (merge) ns = na + nb;
            else if (count || x.op == OP_AND) ns = mn;
            else ns = na;
            if (count) np = 0;
            else if (x.op == OP_OR || x.op == OP_XOR) np = na + nb;
            else if (x.op == OP_ANDNOT) np = na;
            else np = merge ? na : mn;
            d.n_slots = (uint32_t)ns;
            d.n_pos = (uint32_t)np;
            S.small_bound += mn;   // matched keys: at most the smaller key count
            S.ed += 2ull * (A->n_bitsets + B->n_bitsets) + ns / 16;
            if (!count) {
                S.any_mat = true;
                uint64_t w1, b1;
                query_bounds(A, B, x.op, w1, b1);
                S.bw += w1;
                S.bb += b1;
                if (x.op == OP_AND) {
                    S.ew += std::min(A->word_bytes, B->word_bytes);
                    S.eb += 8192ull * std::min(A->n_bitsets, B->n_bitsets);
                } else if (x.op == OP_ANDNOT) {
                    S.ew += A->word_bytes;
                    S.eb += 8192ull * A->n_bitsets;
                } else {
                    S.ew += A->word_bytes + B->word_bytes;
                    S.eb += 8192ull * ((uint64_t)A->n_bitsets + B->n_bitsets);
                }
            }
        }
    });
    uint64_t npos = 0, tiles = 0, ew = 0, eb = 0, bw = 0, bb = 0, ed = 0, small_bound = 0;
    p->meta_bytes = 0;
    for (const Sums &S : part) {
        p->meta_bytes += S.meta;
        small_bound += S.small_bound;
        ed += S.ed;
        ew += S.ew;
        eb += S.eb;
        bw += S.bw;
        bb += S.bb;
        p->any_mat = p->any_mat || S.any_mat;
    }
    for (uint64_t i = 0; i < nq; i++) {
        PairDev &d = p->pairs[i];
        d.pos_base = npos;
        npos += d.n_pos;
        tb[i] = tiles;
        tiles += (d.n_slots + 31) / 32;
    }
    tb[nq] = tiles;
    p->total_pos = npos;
    p->total_tiles = tiles;
    p->defer_cap = std::max<uint64_t>(ed, 4096);
    p->small_cap = small_bound + 2ull * SQCHUNK * lean_warps(p, current_schedule());
    if (use_bounds) {
        p->words_cap = bw;
        p->bits_cap = bb;
    } else {
        p->words_cap = std::min<uint64_t>(bw, ew + ew / 8 + (1ull << 20));
        p->bits_cap = std::min<uint64_t>(bb, eb + eb / 8 + 8192ull * 16);
    }
    // device tables: pool views | pairs | tile prefix | stats | exec state
    const uint64_t o_pool = 0;
    const uint64_t o_pairs = align_up(o_pool + sizeof(BmView) * (uint64_t)pool_n, 256);
    const uint64_t o_qv = align_up(o_pairs + sizeof(PairDev) * nq, 256);
    const uint64_t o_tb = align_up(o_qv + sizeof(QViews) * nq, 256);
    const uint64_t o_ord = align_up(o_tb + 8ull * (nq + 1), 256);
    const uint64_t o_stats = align_up(o_ord + 4ull * std::max<uint64_t>(nq, 1), 256);
    const uint64_t o_es = align_up(o_stats + sizeof(PairStats) * nq, 256);
    p->tables_bytes = o_es + 256;
    p->tables = (uint8_t *)dev_alloc(p->tables_bytes, s);
    if (!p->tables) { plan_destroy(p); return RB_ENOMEM; }
    p->d_pool = (BmView *)(p->tables + o_pool);
    p->d_pairs = (PairDev *)(p->tables + o_pairs);
    p->d_qv = (QViews *)(p->tables + o_qv);
    p->d_tile_base = (unsigned long long *)(p->tables + o_tb);
    p->d_order = (uint32_t *)(p->tables + o_ord);
    p->d_stats = (PairStats *)(p->tables + o_stats);
    p->d_es = (ExecState *)(p->tables + o_es);
    std::vector<uint8_t> hbuf(o_stats);
    BmView *hv = (BmView *)(hbuf.data() + o_pool);
    for (uint32_t i = 0; i < pool_n; i++) hv[i] = view_of(pool[i]);
    if (nq) memcpy(hbuf.data() + o_pairs, p->pairs.data(), sizeof(PairDev) * nq);
    QViews *hq = (QViews *)(hbuf.data() + o_qv);
    parallel_pieces(nq, pieces, [&](uint32_t, uint64_t lo, uint64_t hi) {
        for (uint64_t i = lo; i < hi; i++) hq[i] = {hv[p->pairs[i].a], hv[p->pairs[i].b]};
    });
    memcpy(hbuf.data() + o_tb, tb.data(), 8ull * (nq + 1));
    if (nq < 4096) {
        // k_compact's order: the materialising queries by output slots,
        // largest first, ties in query order
        std::vector<uint32_t> ord;
        ord.reserve(nq);
        for (uint64_t i = 0; i < nq; i++)
            if (!(p->pairs[i].flags & F_COUNT) && p->pairs[i].n_pos) ord.push_back((uint32_t)i);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](uint32_t x, uint32_t y) { return p->pairs[x].n_pos > p->pairs[y].n_pos; });
        p->n_order = (uint32_t)ord.size();
        if (!ord.empty()) memcpy(hbuf.data() + o_ord, ord.data(), 4ull * ord.size());
    } else {
        // the same order for large batches by a counting sort (the slot
        // counts are at most twice the largest key count; a comparison sort
        // of 65,536 queries took 3.6 ms)
        uint32_t top = 0;
        for (uint64_t i = 0; i < nq; i++)
            if (!(p->pairs[i].flags & F_COUNT)) top = std::max(top, p->pairs[i].n_pos);
        std::vector<uint32_t> start((size_t)top + 2, 0);
        for (uint64_t i = 0; i < nq; i++)
            if (!(p->pairs[i].flags & F_COUNT) && p->pairs[i].n_pos) start[top - p->pairs[i].n_pos + 1]++;
        for (size_t v = 1; v < start.size(); v++) start[v] += start[v - 1];
        uint32_t *ord = reinterpret_cast<uint32_t *>(hbuf.data() + o_ord);
        for (uint64_t i = 0; i < nq; i++)
            if (!(p->pairs[i].flags & F_COUNT) && p->pairs[i].n_pos) ord[start[top - p->pairs[i].n_pos]++] = (uint32_t)i;
        p->n_order = start[top];
    }
    cudaError_t e = cudaMallocHost((void **)&p->h_stats, sizeof(PairStats) * std::max<uint64_t>(nq, 1));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&p->h_es, sizeof(ExecState));
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->tables, hbuf.data(), o_stats, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev2);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev3);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        plan_destroy(p);
        return cuda_err(e, "plan setup");
    }
    *out = p;
    return RB_OK;
}

// the launch sequence of one run, enqueued on stream s; when captured, the
// events become external event-record nodes so the kernel times can still
// be read after a graph replay
// warps of the k_heavy launch for this schedule that can take deferred pairs
uint64_t heavy_warps(const rb_plan *p, const rb_schedule &sc) {
    const uint64_t w = (uint64_t)sm_count() * std::max<uint32_t>(1, sc.ctas_per_sm) * sc.warps_per_cta;
    return std::min<uint64_t>(w, p->defer_cap);
}

// warps of the k_lean launch for this plan and schedule
uint64_t lean_warps(const rb_plan *p, const rb_schedule &sc) {
    const unsigned long long lean_cap =
        (unsigned long long)sm_count() * (sc.lean_ctas_per_sm ? sc.lean_ctas_per_sm : LEAN_CTAS_MAX) * (LEAN_THREADS / 32);
    const unsigned long long warps = std::min<unsigned long long>(p->total_tiles, lean_cap);
    return std::max<unsigned long long>(1, (warps + LEAN_THREADS / 32 - 1) / (LEAN_THREADS / 32)) *
           (LEAN_THREADS / 32);
}

cudaError_t enqueue_run(rb_plan *p, const rb_schedule &sc, cudaStream_t s, bool capture) {
    const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
    const uint64_t nq = p->q.size();
    cudaError_t e = cudaMemcpyAsync(p->d_es, p->h_es, sizeof(ExecState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nq) e = cudaMemsetAsync(p->d_stats, 0, sizeof(PairStats) * nq, s);
    if (e != cudaSuccess) return e;
    PairParams P;
    P.pool = p->d_pool;
    P.pairs = p->d_pairs;
    P.qv = p->d_qv;
    P.tile_base = p->d_tile_base;
    P.stats = p->d_stats;
    P.es = p->d_es;
    P.n_tiles = p->total_tiles;
    P.n_pairs = (uint32_t)nq;
    P.small_iv = sc.small_intervals;
    P.prefetch = sc.prefetch_lines;
    // consecutive tiles per take: the schedule's, fewer for small plans so
    // that every lean warp still gets some 64 takes (the last takes of a
    // run are what balances its warps)
    {
        const uint64_t take = sc.tiles_per_take ? sc.tiles_per_take : 32;
        const uint64_t fair = p->total_tiles / (lean_warps(p, sc) * 64);
        P.chunk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(take, fair));
    }
    init_kernel_attrs();
    if ((e = cudaEventRecordWithFlags(p->ev0, s, evf)) != cudaSuccess) return e;
    if (p->total_tiles) {
        const unsigned grid = (unsigned)(lean_warps(p, sc) / (LEAN_THREADS / 32));
        k_lean<<<grid, LEAN_THREADS, 0, s>>>(P);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(p->ev1, s, evf)) != cudaSuccess) return e;
    if (p->total_tiles) {
        const unsigned grid = (unsigned)std::max<uint64_t>(
            1, std::min<uint64_t>((p->small_cap + 31) / 32, (uint64_t)sm_count() * SMALL_CTAS_MAX * (LEAN_THREADS / 32)) /
                   (LEAN_THREADS / 32));
        k_small<<<grid, LEAN_THREADS, 0, s>>>(P);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(p->ev3, s, evf)) != cudaSuccess) return e;
    if (p->total_tiles) {
        switch (sc.warps_per_cta) {
            case 2: launch_heavy_w<2>(P, sc.ctas_per_sm, s); break;
            case 8: launch_heavy_w<8>(P, sc.ctas_per_sm, s); break;
            default: launch_heavy_w<4>(P, sc.ctas_per_sm, s); break;
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(p->ev2, s, evf)) != cudaSuccess) return e;
    if (p->any_mat && p->n_order) {
        unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(p->n_order, (uint64_t)sm_count() * 4));
        k_compact<<<grid, 512, 0, s>>>(p->d_pairs, p->d_order, p->n_order, p->d_stats, p->d_es);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (nq) e = cudaMemcpyAsync(p->h_stats, p->d_stats, sizeof(PairStats) * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_es, p->d_es, sizeof(ExecState), cudaMemcpyDeviceToHost, s);
    return e;
}

struct ArenaLayout {
    uint64_t o_keys, o_defer, o_small, o_words, o_bits, bytes;
    uint64_t words_cap;   // word region incl. the slack of k_lean's per-warp chunks
    uint32_t wchunk;      // bytes of one per-warp word chunk
    uint64_t bits_cap;    // bitset region incl. the slack of k_heavy's per-warp chunks
};

// The per-warp word chunk: the largest power of two in [WCHUNK_MIN,
// WCHUNK_MAX] whose one unfinished chunk per warp stays within 1/16 of the
// word bytes the plan expects (small batches keep small chunks and small
// arenas; large ones refill from the shared counter rarely)
uint32_t word_chunk(uint64_t words, uint64_t warps) {
    uint32_t c = WCHUNK_MAX;
    while (c > WCHUNK_MIN && (uint64_t)c * warps * 16 > words) c >>= 1;
    return c;
}

ArenaLayout arena_layout(const rb_plan *p) {
    ArenaLayout L;
    const uint64_t T = p->total_pos;
    L.o_keys = align_up(8 * T, 256);
    L.o_defer = align_up(L.o_keys + 2 * T, 256);
    L.o_small = align_up(L.o_defer + sizeof(Deferred) * p->defer_cap, 256);
    L.o_words = align_up(L.o_small + sizeof(Item) * p->small_cap, 256);
    const rb_schedule sc = current_schedule();
    const uint64_t warps = lean_warps(p, sc) + heavy_warps(p, sc);
    L.wchunk = word_chunk(p->words_cap, warps);
    L.words_cap = p->words_cap + p->words_cap / 7 + warps * L.wchunk;
    L.o_bits = align_up(L.o_words + L.words_cap, 256);
    L.bits_cap = p->bits_cap + heavy_warps(p, current_schedule()) * (HCHUNK - 1) * 8192ull;
    L.bytes = L.o_bits + L.bits_cap;
    return L;
}

// Enqueue one run with the plan's current caps: as a graph replay on the
// plan's own stream, ordered after the work already on s and with s ordered
// after it, or directly on s.  *arena receives the result memory.
rb_status run_launch(rb_plan *p, cudaStream_t s, bool graph, RbArena **arena) {
    *arena = nullptr;
    const rb_schedule sc = current_schedule();
    const ArenaLayout L = arena_layout(p);
    if (L.bytes >= MAX_OFFSET)
        return set_err(RB_ERANGE, "batch results need %llu bytes, above the 128 GiB descriptor reach; split the batch",
                       (unsigned long long)L.bytes);
    RbArena *a = arena_new(L.bytes, s);
    if (!a) return RB_ENOMEM;
    ExecState &h = *p->h_es;
    memset(&h, 0, sizeof h);
    h.arena = (uint8_t *)a->ptr;
    h.descs = (uint64_t *)a->ptr;
    h.keys = (uint16_t *)((uint8_t *)a->ptr + L.o_keys);
    h.defer = (Deferred *)((uint8_t *)a->ptr + L.o_defer);
    h.defer_cap = p->defer_cap;
    h.small = (Item *)((uint8_t *)a->ptr + L.o_small);
    h.small_cap = p->small_cap;
    h.words_off = L.o_words;
    h.words_cap = L.words_cap;
    h.wchunk = L.wchunk;
    h.bits_off = L.o_bits;
    h.bits_cap = L.bits_cap;
    cudaError_t e = cudaSuccess;
    if (graph) {
        if (!p->ps) e = cudaStreamCreateWithFlags(&p->ps, cudaStreamNonBlocking);
        if (e == cudaSuccess && p->gexec && memcmp(&p->gsched, &sc, sizeof sc) != 0) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        if (e == cudaSuccess && !p->gexec) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(p->ps, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_run(p, sc, p->ps, true);
                e = cudaStreamEndCapture(p->ps, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            p->gsched = sc;
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_in, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->ps, p->ev_in, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(p->gexec, p->ps);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_done, p->ps);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_done, 0);
    } else {
        e = enqueue_run(p, sc, s, false);
    }
    if (e != cudaSuccess) {
        arena_unref(a);
        return cuda_err(e, "batch run");
    }
    *arena = a;
    return RB_OK;
}

// Wait for a launched run and check it.  On success *arena holds the
// results; *overflow tells the caller to retry with the exact sizes now
// recorded (the run's memory is then released).
rb_status run_wait(rb_plan *p, cudaStream_t s, bool graph, RbArena *a, RbArena **arena, bool *overflow) {
    *arena = nullptr;
    *overflow = false;
    ExecState &h = *p->h_es;
    cudaError_t e = cudaStreamSynchronize(graph ? p->ps : s);
    if (e != cudaSuccess) {
        arena_unref(a);
        return cuda_err(e, "batch run");
    }
    float m1 = 0.f, m2 = 0.f, m3 = 0.f;
    if (p->total_tiles && cudaEventElapsedTime(&m1, p->ev0, p->ev1) == cudaSuccess &&
        cudaEventElapsedTime(&m3, p->ev1, p->ev3) == cudaSuccess &&
        cudaEventElapsedTime(&m2, p->ev3, p->ev2) == cudaSuccess) {
        p->last_lean_ms = m1;
        p->last_small_ms = m3;
        p->last_heavy_ms = m2;
        p->last_ms = m1 + m3 + m2;
    } else {
        p->last_ms = p->last_lean_ms = p->last_small_ms = p->last_heavy_ms = 0;
    }
    clear_stale_error();
    if (h.status & 4u) {
        arena_unref(a);
        return set_err(RB_ETIMEOUT, "batch: a bulk-copy wait ran out of its iteration limit");
    }
    if (h.status & 3u) {
        *overflow = true;
        p->words_cap = std::max<uint64_t>(p->words_cap, h.words_used);
        p->bits_cap = std::max<uint64_t>(p->bits_cap, h.bits_used);
        p->defer_cap = std::max<uint64_t>(p->defer_cap, h.defer_n);
        p->small_cap = std::max<uint64_t>(p->small_cap, h.small_n1 + h.small_n2 + 2ull * SQCHUNK * lean_warps(p, current_schedule()));
        arena_unref(a);
        return RB_OK;
    }
    if (!p->exact) {
        p->words_cap = h.words_used;
        p->bits_cap = h.bits_used;
        p->defer_cap = std::max<uint64_t>(h.defer_n, 1);
        // later runs may reserve up to one block more per warp and class
        p->small_cap = h.small_n1 + h.small_n2 + 2ull * SQCHUNK * lean_warps(p, current_schedule());
        p->exact = true;
    }
    p->last_lean_bytes = h.lean_bytes + p->meta_bytes;
    p->last_small_bytes = h.small_bytes;
    p->last_heavy_bytes = h.heavy_bytes;
    p->last_deferred = h.defer_n;
    p->last_small = h.small_n1 + h.small_n2;
    *arena = a;
    return RB_OK;
}

rb_status run_once(rb_plan *p, cudaStream_t s, bool graph, RbArena **arena, bool *overflow) {
    RbArena *a = nullptr;
    rb_status st = run_launch(p, s, graph, &a);
    if (st != RB_OK) return st;
    return run_wait(p, s, graph, a, arena, overflow);
}

rb_status finish_results(rb_plan *p, RbArena *a, rb_t **outs, uint64_t *counts);

// a launched run (first) collected, retried synchronously with the exact
// sizes while the arena overflowed, then turned into results
rb_status plan_complete(rb_plan *p, RbArena *first, rb_t **outs, uint64_t *counts, cudaStream_t s, bool graph) {
    RbArena *a = nullptr;
    bool overflow = false;
    rb_status st = run_wait(p, s, graph, first, &a, &overflow);
    for (int attempt = 1; st == RB_OK && overflow && attempt < 3; attempt++) st = run_once(p, s, false, &a, &overflow);
    if (st != RB_OK) return st;
    if (overflow) return set_err(RB_ENOMEM, "batch: output arena overflow persisted");
    return finish_results(p, a, outs, counts);
}

rb_status plan_execute(rb_plan *p, rb_t **outs, uint64_t *counts, cudaStream_t s, bool graph) {
    clear_stale_error();
    RbArena *first = nullptr;
    rb_status st = run_launch(p, s, graph, &first);
    if (st != RB_OK) return st;
    return plan_complete(p, first, outs, counts, s, graph);
}

// result handles and counts of a completed run whose memory is a
rb_status finish_results(rb_plan *p, RbArena *a, rb_t **outs, uint64_t *counts) {
    const uint64_t nq = p->q.size();
    const ArenaLayout L = arena_layout(p);
    uint64_t alg = 0, outb = 0;
    // the result handles share one allocation and take their arena
    // references in one step
    RbBlock *blk = nullptr;
    uint64_t nm = 0;
    if (outs) {
        for (uint64_t i = 0; i < nq; i++) nm += (p->pairs[i].flags & F_COUNT) ? 0 : 1;
        if (nm) {
            blk = new RbBlock;
            blk->items = new rb[nm]();
            blk->refs.store(nm);
            a->refs.fetch_add((int)nm);
        }
    }
    uint64_t used = 0;
    for (uint64_t i = 0; i < nq; i++) {
        const PairDev &d = p->pairs[i];
        const PairStats &S = p->h_stats[i];
        const rb *A = p->pool[d.a], *B = p->pool[d.b];
        if (d.flags & F_COUNT) {
            const uint64_t inter = S.card;
            uint64_t v;
            switch (d.op) {
                case OP_AND: v = inter; break;
                case OP_OR: v = A->card + B->card - inter; break;
                case OP_ANDNOT: v = A->card - inter; break;
                default: v = A->card + B->card - 2 * inter; break;
            }
            if (counts) counts[i] = v;
            if (outs) outs[i] = nullptr;
            continue;
        }
        outb += S.words + 8192ull * S.nbits + 10ull * S.n_out;
        if (counts) counts[i] = S.card;
        if (outs) {
            rb *h = &blk->items[used++];
            h->n = S.n_out;
            h->card = S.card;
            h->word_bytes = S.words;
            h->n_bitsets = S.nbits;
            h->base = (uint8_t *)a->ptr;
            h->descs = (uint64_t *)a->ptr + d.pos_base;
            h->keys = (uint16_t *)((uint8_t *)a->ptr + L.o_keys) + d.pos_base;
            h->arena = a;
            h->block = blk;
            outs[i] = h;
        }
    }
    p->last_alg = alg + p->h_es->lean_bytes + p->meta_bytes + p->h_es->small_bytes + p->h_es->heavy_bytes;
    p->last_out = outb;
    arena_unref(a);
    return RB_OK;
}

rb_status single(const rb_t *a, const rb_t *b, uint32_t op, uint32_t flags, rb_t **out, uint64_t *count,
                 void *stream) {
    if (!a || !b) return set_err(RB_EINVAL, "NULL bitmap");
    if (op > 3) return set_err(RB_EINVAL, "bad op %u", op);
    const rb_t *pool[2] = {a, b};
    rb_query q = {op, 0, 1, flags};
    rb_plan *p = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rb_status st = plan_build(pool, 2, &q, 1, s, true, &p);
    if (st != RB_OK) return st;
    rb_t *o = nullptr;
    uint64_t c = 0;
    st = plan_execute(p, out ? &o : nullptr, &c, s, false);
    plan_destroy(p);
    if (st != RB_OK) return st;
    if (out) *out = o;
    if (count) *count = c;
    return RB_OK;
}

}  // namespace

extern "C" {

rb_status rb_apply(rb_op op, const rb_t *a, const rb_t *b, rb_t **out, void *stream) {
    if (!out) return set_err(RB_EINVAL, "rb_apply: out is NULL");
    *out = nullptr;
    return single(a, b, (uint32_t)op, 0, out, nullptr, stream);
}
rb_status rb_and(const rb_t *a, const rb_t *b, rb_t **out, void *s) { return rb_apply(RB_AND, a, b, out, s); }
rb_status rb_or(const rb_t *a, const rb_t *b, rb_t **out, void *s) { return rb_apply(RB_OR, a, b, out, s); }
rb_status rb_andnot(const rb_t *a, const rb_t *b, rb_t **out, void *s) { return rb_apply(RB_ANDNOT, a, b, out, s); }
rb_status rb_xor(const rb_t *a, const rb_t *b, rb_t **out, void *s) { return rb_apply(RB_XOR, a, b, out, s); }

rb_status rb_apply_cardinality(rb_op op, const rb_t *a, const rb_t *b, uint64_t *out, void *stream) {
    if (!out) return set_err(RB_EINVAL, "NULL output");
    return single(a, b, (uint32_t)op, RB_Q_COUNT_ONLY, nullptr, out, stream);
}
rb_status rb_and_cardinality(const rb_t *a, const rb_t *b, uint64_t *o, void *s) {
    return rb_apply_cardinality(RB_AND, a, b, o, s);
}
rb_status rb_or_cardinality(const rb_t *a, const rb_t *b, uint64_t *o, void *s) {
    return rb_apply_cardinality(RB_OR, a, b, o, s);
}
rb_status rb_andnot_cardinality(const rb_t *a, const rb_t *b, uint64_t *o, void *s) {
    return rb_apply_cardinality(RB_ANDNOT, a, b, o, s);
}
rb_status rb_xor_cardinality(const rb_t *a, const rb_t *b, uint64_t *o, void *s) {
    return rb_apply_cardinality(RB_XOR, a, b, o, s);
}

rb_status rb_jaccard(const rb_t *a, const rb_t *b, double *out, uint64_t *inter, uint64_t *uni, void *stream) {
    uint64_t i = 0;
    rb_status st = single(a, b, RB_AND, RB_Q_COUNT_ONLY, nullptr, &i, stream);
    if (st != RB_OK) return st;
    const uint64_t u = a->card + b->card - i;
    if (inter) *inter = i;
    if (uni) *uni = u;
    if (out) *out = u ? (double)i / (double)u : 0.0;
    return RB_OK;
}

rb_status rb_batch_op(const rb_t *const *pool, uint32_t pool_n, const rb_query *q, uint64_t nq, rb_t **outs,
                      uint64_t *counts, void *stream) {
    if (outs)
        for (uint64_t i = 0; i < nq; i++) outs[i] = nullptr;
    for (uint64_t i = 0; i < nq && q; i++)
        if (!(q[i].flags & RB_Q_COUNT_ONLY) && !outs)
            return set_err(RB_EINVAL, "rb_batch_op: outs is NULL but query %llu materialises", (unsigned long long)i);
    rb_plan *p = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    rb_status st = plan_build(pool, pool_n, q, nq, s, false, &p);
    if (st != RB_OK) return st;
    st = plan_execute(p, outs, counts, s, false);
    plan_destroy(p);
    return st;
}

rb_status rb_batch_jaccard(const rb_t *const *pool, uint32_t pool_n, const uint32_t *a, const uint32_t *b,
                           uint64_t n, double *jac, uint64_t *inter, uint64_t *uni, void *stream) {
    if (n && (!a || !b)) return set_err(RB_EINVAL, "rb_batch_jaccard: NULL index arrays");
    std::vector<rb_query> q(n);
    for (uint64_t i = 0; i < n; i++) q[i] = {RB_AND, a[i], b[i], RB_Q_COUNT_ONLY};
    std::vector<uint64_t> c(n);
    rb_status st = rb_batch_op(pool, pool_n, q.data(), n, nullptr, c.data(), stream);
    if (st != RB_OK) return st;
    for (uint64_t i = 0; i < n; i++) {
        const uint64_t u = pool[a[i]]->card + pool[b[i]]->card - c[i];
        if (inter) inter[i] = c[i];
        if (uni) uni[i] = u;
        if (jac) jac[i] = u ? (double)c[i] / (double)u : 0.0;
    }
    return RB_OK;
}

rb_status rb_plan_create(const rb_t *const *pool, uint32_t pool_n, const rb_query *q, uint64_t nq, void *stream,
                         rb_plan_t **out) {
    if (!out) return set_err(RB_EINVAL, "rb_plan_create: out is NULL");
    return plan_build(pool, pool_n, q, nq, (cudaStream_t)stream, false, out);
}

rb_status rb_plan_run(rb_plan_t *p, rb_t **outs, uint64_t *counts, void *stream) {
    if (!p) return set_err(RB_EINVAL, "rb_plan_run: NULL plan");
    // a launched run owns the plan's execution state until it is collected
    if (p->pending) return set_err(RB_EINVAL, "rb_plan_run: a launched run has not been collected");
    if (outs)
        for (uint64_t i = 0; i < p->q.size(); i++) outs[i] = nullptr;
    if (p->any_mat && !outs) return set_err(RB_EINVAL, "rb_plan_run: outs is NULL but the plan materialises");
    // the first run sizes the arena exactly; later runs replay a CUDA graph
    return plan_execute(p, outs, counts, (cudaStream_t)stream, p->exact);
}

rb_status rb_plan_launch(rb_plan_t *p, void *stream) {
    if (!p) return set_err(RB_EINVAL, "rb_plan_launch: NULL plan");
    if (p->pending) return set_err(RB_EINVAL, "rb_plan_launch: the previous run has not been collected");
    clear_stale_error();
    RbArena *a = nullptr;
    rb_status st = run_launch(p, (cudaStream_t)stream, p->exact, &a);
    if (st != RB_OK) return st;
    p->pending = a;
    p->pending_graph = p->exact;
    p->pending_stream = (cudaStream_t)stream;
    return RB_OK;
}

rb_status rb_plan_collect(rb_plan_t *p, rb_t **outs, uint64_t *counts) {
    if (!p) return set_err(RB_EINVAL, "rb_plan_collect: NULL plan");
    if (!p->pending) return set_err(RB_EINVAL, "rb_plan_collect: no run was launched");
    if (outs)
        for (uint64_t i = 0; i < p->q.size(); i++) outs[i] = nullptr;
    RbArena *a = p->pending;
    p->pending = nullptr;
    if (p->any_mat && !outs) {
        // the run still has to finish before its memory goes back
        plan_complete(p, a, nullptr, nullptr, p->pending_stream, p->pending_graph);
        return set_err(RB_EINVAL, "rb_plan_collect: outs is NULL but the plan materialises");
    }
    return plan_complete(p, a, outs, counts, p->pending_stream, p->pending_graph);
}

rb_status rb_plan_stats(const rb_plan_t *p, rb_plan_timing *t) {
    if (!p || !t) return set_err(RB_EINVAL, "rb_plan_stats: NULL argument");
    t->lean_ms = p->last_lean_ms;
    t->heavy_ms = p->last_heavy_ms;
    t->lean_bytes = p->last_lean_bytes;
    t->heavy_bytes = p->last_heavy_bytes;
    t->alg_bytes = p->last_alg;
    t->out_bytes = p->last_out;
    t->deferred = p->last_deferred;
    t->small_ms = p->last_small_ms;
    t->small_bytes = p->last_small_bytes;
    t->small_pairs = p->last_small;
    return RB_OK;
}

void rb_plan_free(rb_plan_t *p) { plan_destroy(p); }

rb_status rb_autotune(rb_plan_t *p, uint32_t reps, void *stream, rb_schedule *best, double *best_ms) {
    if (!p) return set_err(RB_EINVAL, "rb_autotune: NULL plan");
    if (p->pending) return set_err(RB_EINVAL, "rb_autotune: a launched run has not been collected");
    if (reps == 0) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    const rb_schedule saved = current_schedule();
    std::vector<rb_t *> outs(p->q.size(), nullptr);
    // mean kernel time of reps runs after one warm-up run (CUDA events on
    // the launching stream, key merge + container-pair stages); < 0 if the
    // schedule does not run
    auto measure = [&](const rb_schedule &c) -> double {
        if (rb_set_schedule(&c) != RB_OK) return -1.0;
        double tot = 0;
        for (uint32_t r = 0; r < reps + 1; r++) {
            const rb_status st = plan_execute(p, outs.data(), nullptr, s, false);
            for (auto &h : outs) { rb_free(h); h = nullptr; }
            if (st != RB_OK) return -1.0;
            if (r > 0) tot += p->last_ms;
        }
        return tot / reps;
    };
    // Coordinate descent from the current schedule over the knobs that
    // change the kernels' speed: the heavy kernel's shape (warps per CTA x
    // CTAs per SM), the largest array pair one lane merges alone (larger
    // ones go to 8-lane groups), the lean kernel's CTAs per SM, the L2
    // prefetch depth and the tiles a lean warp takes at once.  Each pass tries every value of one knob with the
    // others fixed and keeps the fastest; it stops after a pass that
    // changes nothing (at most three passes).
    static const uint32_t heavy[][2] = {{2, 6}, {4, 3}, {8, 1}};
    static const uint32_t smalls[] = {32, 48, 64, 96, 128};
    static const uint32_t leans[] = {6, 7, LEAN_CTAS_MAX};
    static const uint32_t prefs[] = {0, 2, 4, 8};
    static const uint32_t takes[] = {8, 16, 32, 64};
    rb_schedule win = saved;
    if (win.lean_ctas_per_sm == 0) win.lean_ctas_per_sm = LEAN_CTAS_MAX;
    if (win.tiles_per_take == 0) win.tiles_per_take = 32;
    double win_ms = measure(win);
    if (win_ms < 0) win_ms = 1e30;
    auto consider = [&](const rb_schedule &c) -> bool {
        if (memcmp(&c, &win, sizeof c) == 0) return false;
        const double ms = measure(c);
        if (ms >= 0 && ms < win_ms) {
            win_ms = ms;
            win = c;
            return true;
        }
        return false;
    };
    for (int pass = 0; pass < 3; pass++) {
        bool changed = false;
        for (auto &h : heavy) {
            rb_schedule c = win;
            c.warps_per_cta = h[0];
            c.ctas_per_sm = h[1];
            changed |= consider(c);
        }
        for (uint32_t v : smalls) {
            rb_schedule c = win;
            c.small_intervals = v;
            changed |= consider(c);
        }
        for (uint32_t v : leans) {
            rb_schedule c = win;
            c.lean_ctas_per_sm = v;
            changed |= consider(c);
        }
        for (uint32_t v : prefs) {
            rb_schedule c = win;
            c.prefetch_lines = v;
            changed |= consider(c);
        }
        for (uint32_t v : takes) {
            rb_schedule c = win;
            c.tiles_per_take = v;
            changed |= consider(c);
        }
        if (!changed) break;
    }
    rb_set_schedule(win_ms < 1e30 ? &win : &saved);
    if (best) *best = current_schedule();
    if (best_ms) *best_ms = win_ms;
    return win_ms < 1e30 ? RB_OK : set_err(RB_ECUDA, "rb_autotune: no schedule ran");
}

}  // extern "C"
