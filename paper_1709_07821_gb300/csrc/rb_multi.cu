// rb_multi.cu - k-way AND / OR over many bitmaps in one pass (Sec. 5 "Wide
// unions" computes the union of many sets; this engine folds the k
// containers of each output key once, instead of a sequential fold).
//
// Output keys.  AND: the keys of the member with the fewest keys (a key
// survives only if every member has it), in that member's order.  OR: the
// distinct keys of all members in ascending order: output index p is the
// p-th set bit of a per-query 65536-bit presence bitmap, found through the
// prefix of its word popcounts.  Queries of up to MK members work on tiles
// of 32 output keys (fast path below); wider ones on one key per tile.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "rb_device.cuh"
#include "rb_multi.h"

using namespace rbi;
using namespace rbd;

namespace {

struct MultiDev {
    uint32_t op, count_only, k, driver;
    uint32_t mbase, obase, pres_idx, n_slots;
    unsigned long long slot_base;
};

struct MStats {
    unsigned long long card, words, in_bytes;
    unsigned int n_out, n_pos, nbits, pad;
};

struct MState {
    uint8_t *arena;
    uint16_t *keys;
    uint64_t *descs;
    unsigned long long words_off, words_cap, bits_off, bits_cap;
    unsigned long long words_used, bits_used, work;
    unsigned int status, pad;
};

struct MParams {
    const BmView *pool;
    const MultiDev *qs;
    const uint32_t *members;
    const uint32_t *moff;
    const unsigned long long *tile_base;
    const unsigned long long *pres;
    const uint32_t *prefix;
    MStats *stats;
    MState *es;
    unsigned long long n_tiles;
    uint32_t n_q;
    uint32_t chunk;   // consecutive tiles a warp takes at once
};

__device__ __forceinline__ bool find_key(const BmView &V, uint32_t key, uint32_t &j) {
    j = lower_bound16(V.keys, V.n, key);
    return j < V.n && __ldg(V.keys + j) == key;
}

// T0 = T0 op words, words a shared tile or a global bitset
__device__ __forceinline__ void t_apply(uint64_t *T0, const uint64_t *w, uint32_t op, uint32_t lane) {
    ulonglong2 *D = reinterpret_cast<ulonglong2 *>(T0);
    const ulonglong2 *S = reinterpret_cast<const ulonglong2 *>(w);
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        ulonglong2 a = D[32 * k + lane], b = S[32 * k + lane];
        D[32 * k + lane] = make_ulonglong2(apply_op(op, a.x, b.x), apply_op(op, a.y, b.y));
    }
    __syncwarp();
}

__device__ uint64_t alloc_w(MState *es, uint32_t bytes, uint32_t lane) {
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&es->words_used, (unsigned long long)bytes);
    old = __shfl_sync(FULL, old, 0);
    if (old + bytes > es->words_cap) {
        if (lane == 0) atomicOr(&es->status, 1u);
        return ALLOC_FAIL;
    }
    return es->words_off + old;
}
__device__ uint64_t alloc_b(MState *es, uint32_t lane) {
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&es->bits_used, 8192ull);
    old = __shfl_sync(FULL, old, 0);
    if (old + 8192ull > es->bits_cap) {
        if (lane == 0) atomicOr(&es->status, 1u);
        return ALLOC_FAIL;
    }
    return es->bits_off + old;
}

// ------------------------------------------------------------ fast path
// Queries of at most MK members take this path.  A tile is 32 consecutive
// output keys (AND: keys of the member with the fewest keys; OR: ranks in the
// query's key union, read back from its presence bitmap).  Each member's
// containers for those keys are located once per tile: one binary search per
// member for the key range the tile spans, then a coalesced scan of that
// range (or, when a member holds many more keys there, a binary search per
// output key).  A key whose containers are all arrays with at most LCAP
// values in play is then merged by its own lane (OR: one k-way merge of the
// sorted arrays; AND: the smallest array filtered by binary search in the
// others) from its arrays staged in its share of the warp's 8 KB shared
// tile, straight into its output; the other keys are folded by the whole
// warp in that shared tile, as the general path does.
constexpr uint32_t MK = 8;
constexpr uint32_t LCAP = 1024;  // values in play that one lane merges alone (the rest: the warp's folds)
constexpr uint32_t STAGE_WORDS = 2048;   // the warp's tile, shared out to its lanes by a prefix sum
constexpr uint32_t NOIX = 0xFFFFFFFFu;
constexpr uint32_t MKEY_END = 0x10000u;

struct MScratch {
    uint32_t ix[MK][32];       // container of output key `lane` in member i (NOIX: none)
    uint32_t keys[32];         // the tile's output keys (MKEY_END past the last)
    uint32_t lo[MK], hi[MK];   // each member's keys within the tile's key range
    const uint64_t *bp[MK];    // the bitsets of the key being folded
    // what the warp's previous tile leaves to the next one of the same query:
    // its query, the next tile index, and (OR) the presence word of its last key
    uint32_t c_q, c_next, c_word, pad;
};
constexpr uint32_t MCHUNK = 4;   // most consecutive tiles a warp takes at once (large batches)
// one 8 KB tile per warp (lane staging, then the folds) and its scratch;
// 16 warps per SM at 128 registers per thread (a cap of 102 for 20 warps
// spills inside the merges and is slower)
constexpr uint32_t WARP_SMEM = 8192 + sizeof(MScratch);
constexpr int MULTI_WARPS_PER_SM = 16;

// index of the n-th (from 0) set bit of x, n < popcount(x)
__device__ __forceinline__ uint32_t nth_set_bit(uint64_t x, uint32_t n) {
    uint32_t b = 0;
#pragma unroll
    for (uint32_t w = 32; w; w >>= 1) {
        const uint32_t lo = __popcll(x & ((1ull << w) - 1ull));
        if (n >= lo) {
            n -= lo;
            x >>= w;
            b += w;
        }
    }
    return b;
}

// first index in sorted a[0..n) (shared or global memory) holding a value >= v
__device__ __forceinline__ uint32_t lower_bound_gen(const uint16_t *a, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
#pragma unroll 1
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if ((uint32_t)a[m] < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// first index in sorted a[0..n) holding a value >= v
__device__ __forceinline__ uint32_t lower_bound_u16(const uint16_t *a, uint32_t n, uint32_t v) {
    uint32_t lo = 0, hi = n;
#pragma unroll 1
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if ((uint32_t)__ldg(a + m) < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// first index i of sorted keys[0..n) with keys[i] >= key, searched from the
// position key would have if the n keys were spread evenly over [0, 65536):
// a gallop away from that guess brackets the answer, then a binary search
// in the bracket (a few loads for evenly spread keys, O(log n) at worst)
__device__ __forceinline__ uint32_t lower_bound_interp(const uint16_t *keys, uint32_t n, uint32_t key) {
    if (n == 0) return 0;
    uint32_t g = (uint32_t)(((uint64_t)key * n) >> 16);
    if (g >= n) g = n - 1;
    uint32_t lo, hi;   // the answer is in [lo, hi]
    if ((uint32_t)__ldg(keys + g) < key) {
        lo = g + 1;
        hi = n;
        uint32_t step = 1;
#pragma unroll 1
        while (lo + step - 1 < n) {
            if ((uint32_t)__ldg(keys + lo + step - 1) >= key) {
                hi = lo + step - 1;
                break;
            }
            lo += step;
            step <<= 1;
        }
    } else {
        hi = g;
        lo = 0;
        uint32_t step = 1;
#pragma unroll 1
        while (hi >= step) {
            if ((uint32_t)__ldg(keys + hi - step) < key) {
                lo = hi - step + 1;
                break;
            }
            hi -= step;
            step <<= 1;
        }
    }
    return lo + lower_bound16(keys + lo, hi - lo, key);
}

// first index i >= start of sorted keys[0..n) with keys[i] >= key, looking at
// the 32 keys from start first (one or two cache lines) and searching the
// rest only if they are all smaller
__device__ __forceinline__ uint32_t lb_from(const uint16_t *keys, uint32_t n, uint32_t start, uint32_t key) {
    if (start >= n) return n;
    const uint32_t w = min(n - start, 32u);
    const uint32_t r = lower_bound16(keys + start, w, key);
    if (r < w || start + w == n) return start + r;
    return start + w + lower_bound16(keys + start + w, n - start - w, key);
}

// The folds below work on the accumulator tile alone (no second tile), so
// that a warp needs 8 KB of shared memory: word n of a tile holds the values
// [64n, 64n + 64).

// OR: set the bits of every run [s, e] of a run container; AND: clear every
// bit outside its runs (the gaps before, between and after them).  Lanes take
// the ranges in turn; the words a range covers whole are written whole and
// its edge words by atomics (neighbouring ranges can share an edge word,
// never a whole word, since runs are maximal).
template <bool OR>
__device__ void t_runs_inplace(uint64_t *T, const uint32_t *runs, uint32_t r, uint32_t lane) {
    unsigned long long *TU = reinterpret_cast<unsigned long long *>(T);
    const uint32_t n = OR ? r : r + 1;
#pragma unroll 1
    for (uint32_t i = lane; i < n; i += 32) {
        int s, e;   // the range [s, e]; empty when e < s
        if (OR) {
            const uint32_t w = __ldg(runs + i);
            s = (int)(w & 0xFFFFu);
            e = s + (int)(w >> 16);
        } else {
            if (i == 0) {
                s = 0;
            } else {
                const uint32_t w = __ldg(runs + i - 1);
                s = (int)(w & 0xFFFFu) + (int)(w >> 16) + 1;
            }
            e = i == r ? 65535 : (int)(__ldg(runs + i) & 0xFFFFu) - 1;
        }
        if (e < s) continue;
        const uint32_t ws = (uint32_t)s >> 6, we = (uint32_t)e >> 6;
        const unsigned long long ms = ~0ull << (s & 63), me = ~0ull >> (63 - (e & 63));
        if (ws == we) {
            if (OR) atomicOr(TU + ws, ms & me);
            else atomicAnd(TU + ws, ~(ms & me));
            continue;
        }
        if (OR) atomicOr(TU + ws, ms);
        else atomicAnd(TU + ws, ~ms);
#pragma unroll 1
        for (uint32_t w = ws + 1; w < we; w++) TU[w] = OR ? ~0ull : 0ull;
        if (OR) atomicOr(TU + we, me);
        else atomicAnd(TU + we, ~me);
    }
    __syncwarp();
}

// T &= the bits of the sorted array v[0..c): each word is ANDed with the mask
// of the array's values in its stretch; lane l takes words l, l + 32, ...
// (consecutive lanes, consecutive words), finding each word's first value by
// a binary search over the rest of the array from its previous position
__device__ void t_and_array_inplace(uint64_t *T, const uint16_t *v, uint32_t c, uint32_t lane) {
    uint32_t j = 0;
#pragma unroll 1
    for (uint32_t w = lane; w < 1024; w += 32) {
        const uint32_t lo = w << 6;
        j += lower_bound_u16(v + j, c - j, lo);
        uint64_t m = 0;
#pragma unroll 1
        for (; j < c; j++) {
            const uint32_t x = __ldg(v + j);
            if (x >= lo + 64) break;
            m |= 1ull << (x - lo);
        }
        T[w] &= m;
    }
    __syncwarp();
}

// fold one container into the accumulator tile T0 (op: AND or OR)
__device__ void fold_into(uint64_t *T0, const CRef &x, uint32_t op, uint32_t lane) {
    if (x.type == T_BITSET) {
        t_apply(T0, reinterpret_cast<const uint64_t *>(x.p), op, lane);
    } else if (x.type == T_ARRAY) {
        if (op == OP_OR) {
            t_or_array(T0, reinterpret_cast<const uint16_t *>(x.p), x.card, lane);
            __syncwarp();
        } else {
            t_and_array_inplace(T0, reinterpret_cast<const uint16_t *>(x.p), x.card, lane);
        }
    } else if (op == OP_OR) {
        t_runs_inplace<true>(T0, reinterpret_cast<const uint32_t *>(x.p), x.runs, lane);
    } else {
        t_runs_inplace<false>(T0, reinterpret_cast<const uint32_t *>(x.p), x.runs, lane);
    }
}

// run container of r runs from a tile, without scratch: every run start (a
// set bit after a clear one) goes to the low half of its run's output word,
// every run end (a set bit before a clear one) to the high half; a last pass
// turns each word into start | (end - start) << 16
__device__ __noinline__ void t_emit_runs_direct(const uint64_t *T, uint32_t *out, uint32_t r, uint32_t lane) {
    uint16_t *o16 = reinterpret_cast<uint16_t *>(out);
    const ulonglong2 *T2 = reinterpret_cast<const ulonglong2 *>(T);
    uint32_t bs = 0, be = 0, carry = 0;
#pragma unroll 1
    for (int k = 0; k < 16; k++) {
        const ulonglong2 w = T2[32 * k + lane];
        const uint32_t top = (uint32_t)(w.y >> 63);
        uint32_t prev = __shfl_up_sync(FULL, top, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(FULL, top, 31);
        const uint64_t sh0 = (w.x << 1) | (uint64_t)prev, sh1 = (w.y << 1) | (w.x >> 63);
        uint64_t st0 = w.x & ~sh0, st1 = w.y & ~sh1;   // run starts
        uint64_t gs0 = ~w.x & sh0, gs1 = ~w.y & sh1;   // first clear bit after a run
        const uint32_t ns = __popcll(st0) + __popcll(st1), ne = __popcll(gs0) + __popcll(gs1);
        const uint32_t is = warp_incl(ns, lane), ie = warp_incl(ne, lane);
        uint32_t ps = bs + is - ns, pe = be + ie - ne;
        bs += __shfl_sync(FULL, is, 31);
        be += __shfl_sync(FULL, ie, 31);
        const uint32_t v0 = (uint32_t)(64 * k + 2 * lane) * 64u;
        while (st0) { o16[2 * ps++] = (uint16_t)(v0 + __ffsll((long long)st0) - 1); st0 &= st0 - 1; }
        while (st1) { o16[2 * ps++] = (uint16_t)(v0 + 64 + __ffsll((long long)st1) - 1); st1 &= st1 - 1; }
        while (gs0) { o16[2 * pe++ + 1] = (uint16_t)(v0 + __ffsll((long long)gs0) - 2); gs0 &= gs0 - 1; }
        while (gs1) { o16[2 * pe++ + 1] = (uint16_t)(v0 + 64 + __ffsll((long long)gs1) - 2); gs1 &= gs1 - 1; }
    }
    if (carry && lane == 0) o16[2 * be + 1] = 65535;   // the last run reaches the end of the chunk
    __syncwarp();   // the halves written by other lanes are visible from here
#pragma unroll 1
    for (uint32_t i = lane; i < r; i += 32) {
        const uint32_t w = out[i], st = w & 0xFFFFu;
        out[i] = st | ((((w >> 16) - st) & 0xFFFFu) << 16);
    }
    __syncwarp();
}

// T0 = T0 op B_0 op ... op B_{nb-1} over the bitsets at bp[0..nb) (from 0
// instead of T0 when from_zero), counting the result's cardinality c and
// maximal runs r in the same pass; the members' words of a stripe are
// requested four members at a time, so their loads overlap
__device__ __noinline__ void fuse_bitsets(uint64_t *T0, const uint64_t *const *bp, uint32_t nb, uint32_t op,
                                          bool from_zero, uint32_t &c, uint32_t &r, uint32_t lane) {
    ulonglong2 *D = reinterpret_cast<ulonglong2 *>(T0);
    uint32_t cc = 0, rr = 0, carry = 0;
#pragma unroll 1
    for (int k = 0; k < 16; k++) {
        ulonglong2 x = from_zero ? make_ulonglong2(op == OP_AND ? ~0ull : 0ull, op == OP_AND ? ~0ull : 0ull)
                                 : D[32 * k + lane];
        // four members' words requested together (eight at once needed
        // more registers than the kernel's occupancy allows)
#pragma unroll
        for (uint32_t g = 0; g < MK; g += 4) {
            if (g >= nb) break;
            ulonglong2 y[4];
#pragma unroll
            for (uint32_t m = 0; m < 4; m++)
                if (g + m < nb) y[m] = __ldg(reinterpret_cast<const ulonglong2 *>(bp[g + m]) + 32 * k + lane);
#pragma unroll
            for (uint32_t m = 0; m < 4; m++)
                if (g + m < nb) {
                    x.x = apply_op(op, x.x, y[m].x);
                    x.y = apply_op(op, x.y, y[m].y);
                }
        }
        D[32 * k + lane] = x;
        cc += __popcll(x.x) + __popcll(x.y);
        const uint32_t top = (uint32_t)(x.y >> 63);
        uint32_t prev = __shfl_up_sync(FULL, top, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(FULL, top, 31);
        rr += __popcll(x.x & ~((x.x << 1) | (uint64_t)prev)) + __popcll(x.y & ~((x.y << 1) | (x.x >> 63)));
    }
    c = warp_sum(cc);
    r = warp_sum(rr);
    __syncwarp();
}

// after the warp folded one key into T0: count, canonical type, emit, record
__device__ void emit_folded(MState *es, const MultiDev &qd, uint64_t *T0, uint32_t key, uint32_t pos,
                            unsigned long long &card_acc, unsigned long long &words_acc, uint32_t &bits_acc,
                            uint32_t lane, bool counted = false, uint32_t c = 0, uint32_t r = 0) {
    if (!counted) t_combine<false>(nullptr, T0, T0, OP_OR, c, r, lane);
    __syncwarp();
    if (qd.count_only) {
        if (lane == 0) card_acc += c;
        return;
    }
    uint64_t desc = DESC_EMPTY;
    if (c) {
        const uint32_t ty = canon_type(c, r);
        if (ty == T_BITSET) {
            const uint64_t off = alloc_b(es, lane);
            if (off != ALLOC_FAIL) {
                t_emit_bitset(T0, reinterpret_cast<uint64_t *>(es->arena + off), lane);
                desc = mk_desc(c, ty, 0, off);
            }
        } else {
            const uint32_t bytes = word_alloc_bytes(ty, c, r);
            const uint64_t off = alloc_w(es, bytes, lane);
            if (off != ALLOC_FAIL) {
                if (ty == T_ARRAY) {
                    t_emit_array(T0, reinterpret_cast<uint16_t *>(es->arena + off), lane);
                } else {
                    t_emit_runs_direct(T0, reinterpret_cast<uint32_t *>(es->arena + off), r, lane);
                }
                desc = mk_desc(c, ty, ty == T_RUN ? r : 0, off);
            }
        }
    }
    if (lane == 0) {
        es->descs[qd.slot_base + pos] = desc;
        es->keys[qd.slot_base + pos] = (uint16_t)key;
        if (desc != DESC_EMPTY) {
            card_acc += c;
            if (d_type(desc) == T_BITSET) bits_acc++;
            else words_acc += word_alloc_bytes(d_type(desc), c, r);
        }
    }
    __syncwarp();
}

// key of output index p of query q: AND, the p-th key of the member with the
// fewest keys; OR, the p-th key of the union (its presence bitmap and word
// prefix were built by k_presence and k_rank).  False past the last index.
__device__ __forceinline__ bool out_key(const MParams &P, uint32_t q, const MultiDev &qd, const uint32_t *mem,
                                        uint32_t p, uint32_t &key) {
    if (qd.op == OP_AND) {
        if (p >= qd.n_slots) return false;
        key = __ldg(P.pool[mem[qd.driver]].keys + p);
        return true;
    }
    if (p >= P.stats[q].n_pos) return false;
    const uint32_t *pf = P.prefix + (size_t)qd.pres_idx * 1024;
    uint32_t lo = 0, hi = 1024;   // the last word whose prefix is <= p
#pragma unroll 1
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pf[mid] <= p) lo = mid;
        else hi = mid;
    }
    key = lo * 64 + nth_set_bit(P.pres[(size_t)qd.pres_idx * 1024 + lo], p - pf[lo]);
    return true;
}

// Queries of more than MK members (wide unions and intersections): one
// output key per tile.  The warp's lanes search the members for the key 32
// at a time, then the key's containers are folded into T0 one after another
// (AND: only if every member holds the key) and the result is encoded once.
__device__ void multi_key_wide(const MParams &P, uint32_t q, const MultiDev &qd, uint32_t p, uint64_t *T0,
                               uint32_t lane) {
    const uint32_t *mem = P.members + qd.mbase;
    uint32_t key = 0;
    if (!out_key(P, q, qd, mem, p, key)) return;
    MState *es = P.es;
    const bool is_and = qd.op == OP_AND;
    if (is_and) {
        bool absent = false;
#pragma unroll 1
        for (uint32_t i0 = 0; i0 < qd.k && !absent; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t j;
            absent = __any_sync(FULL, i < qd.k && !find_key(P.pool[mem[i]], key, j));
        }
        if (absent) {
            if (!qd.count_only && lane == 0) {
                es->descs[qd.slot_base + p] = DESC_EMPTY;
                es->keys[qd.slot_base + p] = (uint16_t)key;
            }
            return;
        }
    } else {
        t_zero(T0, lane);
        __syncwarp();
    }
    unsigned long long in_acc = 0;
    bool first = true;
#pragma unroll 1
    for (uint32_t i0 = 0; i0 < qd.k; i0 += 32) {
        const uint32_t i = i0 + lane;
        uint64_t d = 0;
        unsigned long long base = 0;
        bool has = false;
        if (i < qd.k) {
            const BmView V = P.pool[mem[i]];
            uint32_t j;
            has = find_key(V, key, j);
            if (has) {
                d = __ldg(V.descs + j);
                base = (unsigned long long)V.base;
            }
        }
        uint32_t m = __ballot_sync(FULL, has);
#pragma unroll 1
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t ds = __shfl_sync(FULL, d, src);
            const CRef x = cref(reinterpret_cast<const uint8_t *>(__shfl_sync(FULL, base, src)), ds);
            in_acc += in_payload_bytes(ds) + 15;
            if (is_and && first) t_decode(T0, x, lane);
            else fold_into(T0, x, qd.op, lane);
            first = false;
        }
    }
    unsigned long long card_acc = 0, words_acc = 0;
    uint32_t bits_acc = 0;
    emit_folded(es, qd, T0, key, p, card_acc, words_acc, bits_acc, lane);
    if (lane == 0) {
        MStats *S = P.stats + q;
        if (card_acc) atomicAdd(&S->card, card_acc);
        if (words_acc) atomicAdd(&S->words, words_acc);
        if (bits_acc) atomicAdd(&S->nbits, bits_acc);
        if (in_acc) atomicAdd(&S->in_bytes, in_acc);
    }
    __syncwarp();
}

// One lane's key, merged from its members' arrays staged one after another
// (each padded to whole words) in the warp's tile S from element sbase on.
// EMIT = false counts the result's values n and maximal runs r; with EMIT
// the result is written to out (4-byte aligned) as type ty: an array as
// pairs of values per word (zero-padded), runs as start | (length - 1) << 16.
// The first pass of a key writes the array form while it counts; only a key
// whose canonical type turns out to be runs is merged a second time.  Each
// member's state is its cursor and end in S and its head value.

// OR: the union of the K members' sorted arrays (the containers MS->ix
// names); each output value takes the smallest head and advances every
// member that holds it
template <uint32_t K, bool EMIT>
__device__ __forceinline__ void kway_union(const MParams &P, const uint32_t *mem, const MScratch *MS, uint32_t lane,
                                           const uint16_t *S, uint32_t sbase, uint32_t ty, uint8_t *out, uint32_t &n,
                                           uint32_t &r) {
    uint32_t at[K], end[K], head[K], w = sbase;
#pragma unroll
    for (uint32_t i = 0; i < K; i++) {
        at[i] = end[i] = w;
        head[i] = MKEY_END;
        const uint32_t j = MS->ix[i][lane];
        if (j != NOIX) {
            const uint32_t len = d_card(__ldg(P.pool[mem[i]].descs + j));
            end[i] = w + len;
            head[i] = S[w];
            w += (len + 1) & ~1u;
        }
    }
    uint32_t *o32 = reinterpret_cast<uint32_t *>(out);
    uint32_t last = 0xFFFFFFFEu, rs = 0, pend = 0;
    n = 0;
    r = 0;
    for (;;) {
        uint32_t v = MKEY_END;
#pragma unroll
        for (uint32_t i = 0; i < K; i++) v = min(v, head[i]);
        if (v == MKEY_END) break;
        if (v != last + 1) {   // a run starts at v
            if (EMIT && ty == T_RUN && r) o32[r - 1] = rs | ((last - rs) << 16);
            rs = v;
            r++;
        }
        if (EMIT && ty == T_ARRAY) {
            if (n & 1) o32[n >> 1] = pend | (v << 16);
            else pend = v;
        }
        n++;
        last = v;
#pragma unroll
        for (uint32_t i = 0; i < K; i++)
            if (head[i] == v) {
                at[i]++;
                head[i] = at[i] < end[i] ? (uint32_t)S[at[i]] : MKEY_END;
            }
    }
    if (EMIT && n) {
        if (ty == T_RUN) o32[r - 1] = rs | ((last - rs) << 16);
        else if (n & 1) o32[n >> 1] = pend;
    }
}

// AND: the values of the smallest array (member min_i) that every other
// member holds, each found by a binary search from that member's cursor
template <uint32_t K, bool EMIT>
__device__ __forceinline__ void and_filter(const MParams &P, const uint32_t *mem, const MScratch *MS, uint32_t min_i,
                                           uint32_t lane, const uint16_t *S, uint32_t sbase, uint32_t ty,
                                           uint8_t *out, uint32_t &n, uint32_t &r) {
    uint32_t at[K], end[K], a0 = 0, n0 = 0, w = sbase;
#pragma unroll
    for (uint32_t i = 0; i < K; i++) {
        const uint32_t len = d_card(__ldg(P.pool[mem[i]].descs + MS->ix[i][lane]));
        at[i] = w;
        end[i] = w + len;
        if (i == min_i) {
            a0 = w;
            n0 = len;
        }
        w += (len + 1) & ~1u;
    }
    uint32_t *o32 = reinterpret_cast<uint32_t *>(out);
    uint32_t last = 0xFFFFFFFEu, rs = 0, pend = 0;
    n = 0;
    r = 0;
    bool more = true;   // false once some member has no value left above the current one
#pragma unroll 1
    for (uint32_t e = 0; e < n0 && more; e++) {
        const uint32_t v = S[a0 + e];
        bool keep = true;
#pragma unroll
        for (uint32_t i = 0; i < K; i++) {
            if (i == min_i || !keep) continue;
            at[i] += lower_bound_gen(S + at[i], end[i] - at[i], v);
            keep = at[i] < end[i] && S[at[i]] == v;
            more = more && at[i] < end[i];
        }
        if (!keep) continue;
        if (v != last + 1) {
            if (EMIT && ty == T_RUN && r) o32[r - 1] = rs | ((last - rs) << 16);
            rs = v;
            r++;
        }
        if (EMIT && ty == T_ARRAY) {
            if (n & 1) o32[n >> 1] = pend | (v << 16);
            else pend = v;
        }
        n++;
        last = v;
    }
    if (EMIT && n) {
        if (ty == T_RUN) o32[r - 1] = rs | ((last - rs) << 16);
        else if (n & 1) o32[n >> 1] = pend;
    }
}

template <bool EMIT>
__device__ __forceinline__ void lane_key(const MParams &P, const uint32_t *mem, const MScratch *MS, uint32_t k,
                                         bool is_and, uint32_t min_i, uint32_t lane, const uint16_t *S,
                                         uint32_t sbase, uint32_t ty, uint8_t *out, uint32_t &n, uint32_t &r) {
    if (is_and) {
        switch (k) {
            case 1: and_filter<1, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            case 2: and_filter<2, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            case 3: and_filter<3, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            case 4: and_filter<4, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            case 5: and_filter<5, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            case 6: and_filter<6, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            case 7: and_filter<7, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
            default: and_filter<8, EMIT>(P, mem, MS, min_i, lane, S, sbase, ty, out, n, r); break;
        }
        return;
    }
    switch (k) {
        case 1: kway_union<1, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        case 2: kway_union<2, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        case 3: kway_union<3, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        case 4: kway_union<4, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        case 5: kway_union<5, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        case 6: kway_union<6, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        case 7: kway_union<7, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
        default: kway_union<8, EMIT>(P, mem, MS, lane, S, sbase, ty, out, n, r); break;
    }
}

__device__ void multi_tile_fast(const MParams &P, uint32_t q, const MultiDev &qd, uint32_t local, uint64_t *T0,
                                MScratch *MS, uint32_t lane) {
    const uint32_t *mem = P.members + qd.mbase;
    const uint32_t k = qd.k;
    const uint32_t p0 = local * 32u;
    const bool cont = MS->c_q == q && MS->c_next == local;   // the previous tile of this warp precedes this one
    uint32_t key = MKEY_END;
    const uint32_t pos = p0 + lane;
    bool valid;
    if (qd.op == OP_AND) {
        valid = out_key(P, q, qd, mem, pos, key);
    } else {
        // OR: the word of the presence bitmap holding the pos-th key, searched
        // in a window of 32 words that starts at the previous tile's last
        // word (or at the word of p0, found by a 32-ary search)
        const uint32_t npos = P.stats[q].n_pos;
        valid = pos < npos;
        if (p0 >= npos) return;
        const uint32_t *pf = P.prefix + (size_t)qd.pres_idx * 1024;
        uint32_t w0 = cont ? MS->c_word : 0;
        if (!cont) {
            uint32_t m = __ballot_sync(FULL, pf[32 * lane] <= p0);
            const uint32_t b = 31 - __clz(m);
            m = __ballot_sync(FULL, pf[32 * b + lane] <= p0);
            w0 = 32 * b + 31 - __clz(m);
        }
        const uint32_t pw = w0 + lane < 1024 ? pf[w0 + lane] : 0xFFFFFFFFu;
        uint32_t j = 0;   // the last window word whose prefix is <= pos
#pragma unroll
        for (uint32_t st = 16; st; st >>= 1)
            if (__shfl_sync(FULL, pw, j + st) <= pos) j += st;
        uint32_t w = w0 + j;
        if (valid && j == 31 && w0 + 32 < 1024 && pf[w0 + 32] <= pos) {   // past the window
            uint32_t lo = w0 + 32, hi = 1024;
#pragma unroll 1
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (pf[mid] <= pos) lo = mid;
                else hi = mid;
            }
            w = lo;
        }
        if (valid) key = w * 64 + nth_set_bit(P.pres[(size_t)qd.pres_idx * 1024 + w], pos - pf[w]);
    }
    const uint32_t n_act = __popc(__ballot_sync(FULL, valid));   // valid lanes are a prefix
    if (n_act == 0) return;
    MS->keys[lane] = key;
    __syncwarp();
    const uint32_t k_lo = MS->keys[0], k_hi = MS->keys[n_act - 1];
    if (lane < k) {
        // each member's keys in [k_lo, k_hi]: continuing tiles start where the
        // previous tile's range ended
        const BmView V = P.pool[mem[lane]];
        const uint32_t lo = cont ? lb_from(V.keys, V.n, MS->hi[lane], k_lo) : lower_bound_interp(V.keys, V.n, k_lo);
        MS->lo[lane] = lo;
        MS->hi[lane] = lb_from(V.keys, V.n, lo, k_hi + 1);
    }
    if (lane == n_act - 1) {
        MS->c_q = q;
        MS->c_next = local + 1;
        MS->c_word = key >> 6;
    }
    for (uint32_t i = 0; i < k; i++) MS->ix[i][lane] = NOIX;
    __syncwarp();
    // locate every member's container of each output key
#pragma unroll 1
    for (uint32_t i = 0; i < k; i++) {
        const BmView V = P.pool[mem[i]];
        const uint32_t lo = MS->lo[i], hi = MS->hi[i];
        if (hi - lo <= 64) {
#pragma unroll 1
            for (uint32_t x0 = lo; x0 < hi; x0 += 32) {
                const uint32_t x = x0 + lane;
                if (x < hi) {
                    const uint32_t kk = __ldg(V.keys + x);
                    uint32_t a = 0, b = n_act;   // first output key >= kk
#pragma unroll 1
                    while (a < b) {
                        const uint32_t m = (a + b) >> 1;
                        if (MS->keys[m] < kk) a = m + 1;
                        else b = m;
                    }
                    if (a < n_act && MS->keys[a] == kk) MS->ix[i][a] = x;
                }
            }
        } else if (lane < n_act) {
            const uint32_t j = lo + lower_bound16(V.keys + lo, hi - lo, key);
            if (j < hi && __ldg(V.keys + j) == key) MS->ix[i][lane] = j;
        }
    }
    __syncwarp();
    // what each output key needs
    MState *es = P.es;
    const bool is_and = qd.op == OP_AND;
    uint32_t present = 0, sum_card = 0, min_card = 0xFFFFFFFFu, min_i = 0;
    bool all_arr = true;
    unsigned long long in_acc = 0;
    if (lane < n_act) {
        for (uint32_t i = 0; i < k; i++) {
            const uint32_t j = MS->ix[i][lane];
            if (j == NOIX) continue;
            const uint64_t d = __ldg(P.pool[mem[i]].descs + j);
            present++;
            sum_card += d_card(d);
            if (d_card(d) < min_card) { min_card = d_card(d); min_i = i; }
            all_arr = all_arr && d_type(d) == T_ARRAY;
            in_acc += in_payload_bytes(d) + 15;
        }
    }
    const bool empty = lane < n_act && is_and && present < k;
    const bool cand = lane < n_act && !empty && all_arr && (is_and ? min_card <= LCAP : sum_card <= LCAP);
    if (empty && !qd.count_only) {
        es->descs[qd.slot_base + pos] = DESC_EMPTY;
        es->keys[qd.slot_base + pos] = (uint16_t)key;
    }
    if (empty) in_acc = 0;   // an absent container ends the key's AND: nothing is read
    // lane path: the key merged by its own lane from its arrays staged in the
    // warp's tile, packed lane after lane by a prefix sum of their words
    // (every lane's words requested at once with cp.async; consecutive lanes
    // start in different banks).  The lanes whose words fit are staged and
    // merged, then the rest in further rounds (the first waiting lane always
    // fits, so each round serves at least one); only a key whose arrays alone
    // pass the tile's size goes to the warp path.  A materialised key is
    // written straight to its output, reserved for the whole tile before the
    // rounds at the size of each key's largest possible array (within the
    // batch's output bound), while it is counted.
    const uint16_t *stage = reinterpret_cast<const uint16_t *>(T0);
    uint32_t words = 0;
    if (cand)
        for (uint32_t i = 0; i < k; i++) {
            const uint32_t j = MS->ix[i][lane];
            if (j != NOIX) words += (d_card(__ldg(P.pool[mem[i]].descs + j)) + 1) / 2;
        }
    const bool lane_path = cand && words <= STAGE_WORDS;
    const bool warp_path = lane < n_act && !empty && !lane_path;
    unsigned long long card_acc = 0, words_acc = 0;
    uint32_t bits_acc = 0;
    uint32_t bytes = 0, oincl = 0;
    uint64_t obase = ALLOC_FAIL;
    if (lane_path && !qd.count_only) bytes = (2 * (is_and ? min_card : sum_card) + 3) & ~3u;
    if (!qd.count_only && __any_sync(FULL, lane_path)) {
        oincl = warp_incl(bytes, lane);
        const uint32_t total = __shfl_sync(FULL, oincl, 31);
        if (total) obase = alloc_w(es, total, lane);
    }
    bool pending = lane_path;
#pragma unroll 1
    while (__any_sync(FULL, pending)) {
        const uint32_t wincl = warp_incl(pending ? words : 0u, lane);
        const bool now = pending && wincl <= STAGE_WORDS;
        uint32_t sbase = 0;
        if (now) {
            uint32_t *S = reinterpret_cast<uint32_t *>(T0) + (wincl - words);
            uint32_t w = 0;
            for (uint32_t i = 0; i < k; i++) {
                const uint32_t j = MS->ix[i][lane];
                if (j == NOIX) continue;
                const BmView V = P.pool[mem[i]];
                const uint64_t d = __ldg(V.descs + j);
                const uint32_t *src = reinterpret_cast<const uint32_t *>(V.base + d_off(d));
                const uint32_t nw = (d_card(d) + 1) / 2;
#pragma unroll 1
                for (uint32_t x = 0; x < nw; x++) cp_async4(S + w + x, src + x);
                w += nw;
            }
            sbase = 2 * (wincl - words);
        }
        cp_async_wait_all();
        __syncwarp();
        if (now) {
            uint32_t n = 0, r = 0;
            if (qd.count_only) {
                lane_key<false>(P, mem, MS, k, is_and, min_i, lane, stage, sbase, 0, nullptr, n, r);
                card_acc += n;
            } else {
                uint64_t desc = DESC_EMPTY;
                if (obase != ALLOC_FAIL) {
                    const uint64_t off = obase + oincl - bytes;
                    lane_key<true>(P, mem, MS, k, is_and, min_i, lane, stage, sbase, T_ARRAY, es->arena + off, n, r);
                    if (n) {
                        const uint32_t ty = canon_type(n, r);   // n <= LCAP <= 4096: array or runs
                        if (ty == T_RUN) {
                            uint32_t n2, r2;
                            lane_key<true>(P, mem, MS, k, is_and, min_i, lane, stage, sbase, T_RUN, es->arena + off,
                                           n2, r2);
                        }
                        desc = mk_desc(n, ty, ty == T_RUN ? r : 0, off);
                        card_acc += n;
                        words_acc += word_alloc_bytes(ty, n, r);
                    }
                }
                es->descs[qd.slot_base + pos] = desc;
                es->keys[qd.slot_base + pos] = (uint16_t)key;
            }
        }
        __syncwarp();   // the tile is staged again in the next round
        pending = pending && !now;
    }
    // warp path: one key at a time in the tile
    uint32_t wl = __ballot_sync(FULL, warp_path);
    while (wl) {
        const int src = __ffs(wl) - 1;
        wl &= wl - 1;
        const uint32_t k_key = __shfl_sync(FULL, key, src), k_pos = __shfl_sync(FULL, pos, src);
        // arrays and runs are folded into T0 one by one (AND starts from the
        // first of them); the bitsets are combined in one pass at the end,
        // which also counts the result
        uint32_t nb = 0;
        bool started = false;
        for (uint32_t i = 0; i < k; i++) {
            const uint32_t j = MS->ix[i][src];
            if (j == NOIX) continue;
            const BmView V = P.pool[mem[i]];
            const CRef x = cref(V.base, __ldg(V.descs + j));
            if (x.type == T_BITSET) {
                if (lane == 0) MS->bp[nb] = reinterpret_cast<const uint64_t *>(x.p);
                nb++;
            } else if (!started) {
                if (is_and) {
                    t_decode(T0, x, lane);
                } else {
                    t_zero(T0, lane);
                    __syncwarp();
                    fold_into(T0, x, OP_OR, lane);
                }
                started = true;
            } else {
                fold_into(T0, x, is_and ? OP_AND : OP_OR, lane);
            }
        }
        __syncwarp();
        uint32_t c = 0, r = 0;
        if (nb) {
            fuse_bitsets(T0, MS->bp, nb, is_and ? OP_AND : OP_OR, !started, c, r, lane);
            emit_folded(es, qd, T0, k_key, k_pos, card_acc, words_acc, bits_acc, lane, true, c, r);
        } else {
            emit_folded(es, qd, T0, k_key, k_pos, card_acc, words_acc, bits_acc, lane);
        }
    }
    // per-query sums
    card_acc = warp_sum64(card_acc);
    words_acc = warp_sum64(words_acc);
    in_acc = warp_sum64(in_acc);
    bits_acc = warp_sum(bits_acc);
    if (lane == 0) {
        MStats *S = P.stats + q;
        if (card_acc) atomicAdd(&S->card, card_acc);
        if (words_acc) atomicAdd(&S->words, words_acc);
        if (bits_acc) atomicAdd(&S->nbits, bits_acc);
        if (in_acc) atomicAdd(&S->in_bytes, in_acc);
    }
    __syncwarp();
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, MULTI_WARPS_PER_SM / WARPS) k_multi(MParams P) {
    extern __shared__ __align__(16) uint64_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *T0 = smem + (size_t)warp * (WARP_SMEM / 8);
    MScratch *MS = reinterpret_cast<MScratch *>(T0 + 1024);
    if (lane == 0) MS->c_q = 0xFFFFFFFFu;
    __syncwarp();
    unsigned long long t = 0, t_end = 0, q_lo = 0, q_hi = 0;
    uint32_t q = 0;
    for (;;) {
        if (t == t_end) {
            if (lane == 0) t = atomicAdd(&P.es->work, (unsigned long long)P.chunk);
            t = __shfl_sync(FULL, t, 0);
            if (t >= P.n_tiles) break;
            t_end = min(t + P.chunk, P.n_tiles);
        }
        if (t < q_lo || t >= q_hi) {
            uint32_t lo = 0, hi = P.n_q;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (P.tile_base[mid] <= t) lo = mid;
                else hi = mid;
            }
            q = lo;
            q_lo = P.tile_base[lo];
            q_hi = P.tile_base[lo + 1];
        }
        const MultiDev qd = P.qs[q];
        const uint32_t local = (uint32_t)(t - q_lo);
        if (qd.k <= MK) multi_tile_fast(P, q, qd, local, T0, MS, lane);
        else multi_key_wide(P, q, qd, local, T0, lane);
        __syncwarp();
        t++;
    }
}

// presence bits of every key of every member of every OR query
__global__ void k_presence(const BmView *pool, const MultiDev *qs, const uint32_t *members, const uint32_t *items,
                           uint32_t n_items, unsigned long long *pres) {
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint32_t q = items[2 * it], i = items[2 * it + 1];
        const MultiDev qd = qs[q];
        const BmView V = pool[members[qd.mbase + i]];
        unsigned long long *pr = pres + (size_t)qd.pres_idx * 1024;
        for (uint32_t j = threadIdx.x; j < V.n; j += blockDim.x) {
            const uint32_t key = __ldg(V.keys + j);
            atomicOr(pr + (key >> 6), 1ull << (key & 63));
        }
    }
}

// exclusive prefix of the word popcounts of each OR query's presence bitmap
__global__ void __launch_bounds__(1024) k_rank(const MultiDev *qs, const uint32_t *or_q, uint32_t n_or,
                                               const unsigned long long *pres, uint32_t *prefix, MStats *stats) {
    __shared__ uint32_t s[32];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (uint32_t x = blockIdx.x; x < n_or; x += gridDim.x) {
        const uint32_t q = or_q[x];
        const uint32_t pi = qs[q].pres_idx;
        const uint32_t c = __popcll(pres[(size_t)pi * 1024 + t]);
        const uint32_t inc = warp_incl(c, lane);
        if (lane == 31) s[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = s[lane], vi = warp_incl(v, lane);
            s[lane] = vi - v;
            if (lane == 31) stats[q].n_pos = vi;
        }
        __syncthreads();
        prefix[(size_t)pi * 1024 + t] = s[warp] + inc - c;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(512) k_mcompact(const MultiDev *qs, uint32_t n_q, MStats *stats, const MState *es) {
    __shared__ uint32_t s_w[16];
    __shared__ uint32_t s_tot;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (uint32_t q = blockIdx.x; q < n_q; q += gridDim.x) {
        const MultiDev qd = qs[q];
        if (qd.count_only) continue;
        const uint32_t n = qd.op == OP_OR ? stats[q].n_pos : qd.n_slots;
        uint64_t *D = es->descs + qd.slot_base;
        uint16_t *K = es->keys + qd.slot_base;
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
                const uint32_t v = lane < nw ? s_w[lane] : 0, inc = warp_incl(v, lane);
                if (lane < nw) s_w[lane] = inc - v;
                if (lane == 31) s_tot = inc;
            }
            __syncthreads();
            if (f) {
                const uint32_t at = out + s_w[warp] + __popc(m & lanemask_lt(lane));
                D[at] = d;
                K[at] = k;
            }
            out += s_tot;
            __syncthreads();
        }
        if (tid == 0) stats[q].n_out = out;
    }
}

}  // namespace

namespace rbi {

struct MultiBatch {
    std::vector<const rb *> pool;
    std::vector<MultiDev> qd;
    std::vector<uint32_t> or_q;
    uint64_t total_slots = 0, total_tiles = 0, words_cap = 0, bits_cap = 0;
    uint32_t n_or = 0, n_items = 0;
    bool any_mat = false;
    const BmView *d_pool = nullptr;
    uint8_t *tables = nullptr;
    uint64_t tables_bytes = 0;
    MultiDev *d_qs = nullptr;
    uint32_t *d_members = nullptr, *d_moff = nullptr, *d_items = nullptr, *d_orq = nullptr, *d_prefix = nullptr;
    unsigned long long *d_tb = nullptr, *d_pres = nullptr;
    MStats *d_stats = nullptr;
    MState *d_es = nullptr;
    MStats *h_stats = nullptr;
    MState *h_es = nullptr;
    uint8_t *hpin = nullptr;
    bool native = false;
    uint64_t o_keys = 0, o_words = 0, o_bits = 0, arena_bytes = 0;
};

static void query_bounds(const rb *const *pool, const MultiQuery &x, uint64_t &ns, uint64_t &wcap, uint64_t &bcap) {
    uint64_t sum_n = 0, sum_card = 0, min_card = ~0ull, nmin = ~0ull;
    for (uint32_t m : x.members) {
        const rb *B = pool[m];
        sum_n += B->n;
        sum_card += B->card;
        min_card = std::min(min_card, B->card);
        nmin = std::min<uint64_t>(nmin, B->n);
    }
    if (x.members.empty()) { nmin = 0; min_card = 0; }
    // a canonical container is at most 8192 bytes and at most twice its
    // cardinality (+ 4 bytes of rounding); a bitset needs more than 4096 values
    if (x.op == OP_AND) {
        ns = nmin;
        wcap = std::min<uint64_t>(8192ull * ns, 2 * min_card + 4 * ns);
        bcap = 8192ull * std::min<uint64_t>(ns, min_card / 4097 + 1);
    } else {
        ns = sum_n;
        wcap = std::min<uint64_t>(8192ull * ns, 2 * sum_card + 4 * ns);
        bcap = 8192ull * std::min<uint64_t>(ns, sum_card / 4097 + 1);
    }
}

uint64_t multi_query_bound(const rb *const *pool, const MultiQuery &q) {
    if (q.count_only) return 0;
    uint64_t ns, w, b;
    query_bounds(pool, q, ns, w, b);
    return 10 * ns + w + b + 1024;
}

rb_status multi_prepare(const rb *const *pool, const BmView *d_pool, uint32_t pool_n, const std::vector<MultiQuery> &qs,
                        cudaStream_t s, MultiBatch **out, uint64_t *arena_bytes, PinnedBuf *stage, bool native) {
    *out = nullptr;
    MultiBatch *b = new MultiBatch;
    b->pool.assign(pool, pool + pool_n);
    b->d_pool = d_pool;
    const uint32_t nq = (uint32_t)qs.size();
    b->qd.resize(nq);
    std::vector<uint32_t> members, moff, items;
    std::vector<unsigned long long> tb(nq + 1);
    uint64_t slots = 0, tiles = 0, wcap = 0, bcap = 0;
    for (uint32_t q = 0; q < nq; q++) {
        const MultiQuery &x = qs[q];
        MultiDev &d = b->qd[q];
        memset(&d, 0, sizeof d);
        if (x.op != OP_AND && x.op != OP_OR) {
            delete b;
            return set_err(RB_EINVAL, "multi-way op must be AND or OR");
        }
        d.op = x.op;
        d.count_only = x.count_only ? 1 : 0;
        d.k = (uint32_t)x.members.size();
        d.mbase = (uint32_t)members.size();
        d.obase = (uint32_t)moff.size();
        uint64_t ns = 0, nmin = ~0ull;
        for (uint32_t i = 0; i < d.k; i++) {
            const uint32_t m = x.members[i];
            if (m >= pool_n || !pool[m]) {
                delete b;
                return set_err(RB_EINVAL, "multi-way member %u out of range", m);
            }
            members.push_back(m);
            moff.push_back((uint32_t)ns);
            const rb *B = pool[m];
            ns += B->n;
            if (B->n < nmin) { nmin = B->n; d.driver = i; }
        }
        moff.push_back((uint32_t)ns);
        uint64_t qw = 0, qb = 0;
        query_bounds(pool, x, ns, qw, qb);
        d.n_slots = (uint32_t)ns;
        if (d.op == OP_OR && d.k) {
            d.pres_idx = b->n_or++;
            b->or_q.push_back(q);
            for (uint32_t i = 0; i < d.k; i++) { items.push_back(q); items.push_back(i); }
        }
        if (!d.count_only) {
            b->any_mat = true;
            d.slot_base = slots;
            slots += ns;
            wcap += qw;
            bcap += qb;
        }
        tb[q] = tiles;
        // fast path: 32 output keys per tile; wide queries: one (the union has
        // at most 65536 keys)
        tiles += d.k <= MK ? (ns + 31) / 32 : (d.op == OP_OR ? std::min<uint64_t>(ns, 65536) : ns);
    }
    tb[nq] = tiles;
    b->n_items = (uint32_t)(items.size() / 2);
    b->total_slots = slots;
    b->total_tiles = tiles;
    b->words_cap = wcap;
    b->bits_cap = bcap;
    b->o_keys = align_up(8 * slots, 256);
    b->o_words = align_up(b->o_keys + 2 * slots, 256);
    b->o_bits = align_up(b->o_words + wcap, 256);
    b->arena_bytes = b->any_mat ? std::max<uint64_t>(256, b->o_bits + bcap) : 0;
    if (b->arena_bytes >= MAX_OFFSET) {
        delete b;
        return set_err(RB_ERANGE, "multi-way results bound above the 128 GiB descriptor reach");
    }
    // device tables
    const uint64_t o_qs = 0;
    const uint64_t o_mem = align_up(o_qs + sizeof(MultiDev) * nq, 256);
    const uint64_t o_moff = align_up(o_mem + 4 * members.size(), 256);
    const uint64_t o_items = align_up(o_moff + 4 * moff.size(), 256);
    const uint64_t o_orq = align_up(o_items + 4 * items.size(), 256);
    const uint64_t o_tb = align_up(o_orq + 4 * b->or_q.size(), 256);
    const uint64_t o_up = align_up(o_tb + 8ull * (nq + 1), 256);   // end of uploaded part
    const uint64_t o_pres = o_up;
    const uint64_t o_prefix = align_up(o_pres + 8192ull * b->n_or, 256);
    const uint64_t o_stats = align_up(o_prefix + 4096ull * b->n_or, 256);
    const uint64_t o_es = align_up(o_stats + sizeof(MStats) * nq, 256);
    b->tables_bytes = o_es + 256;
    b->native = native;
    b->tables = (uint8_t *)(native ? dev_alloc_native(b->tables_bytes, s) : dev_alloc(b->tables_bytes, s));
    if (!b->tables) { delete b; return RB_ENOMEM; }
    b->d_qs = (MultiDev *)(b->tables + o_qs);
    b->d_members = (uint32_t *)(b->tables + o_mem);
    b->d_moff = (uint32_t *)(b->tables + o_moff);
    b->d_items = (uint32_t *)(b->tables + o_items);
    b->d_orq = (uint32_t *)(b->tables + o_orq);
    b->d_tb = (unsigned long long *)(b->tables + o_tb);
    b->d_pres = (unsigned long long *)(b->tables + o_pres);
    b->d_prefix = (uint32_t *)(b->tables + o_prefix);
    b->d_stats = (MStats *)(b->tables + o_stats);
    b->d_es = (MState *)(b->tables + o_es);
    std::vector<uint8_t> h(o_up, 0);
    if (nq) memcpy(h.data() + o_qs, b->qd.data(), sizeof(MultiDev) * nq);
    if (!members.empty()) memcpy(h.data() + o_mem, members.data(), 4 * members.size());
    if (!moff.empty()) memcpy(h.data() + o_moff, moff.data(), 4 * moff.size());
    if (!items.empty()) memcpy(h.data() + o_items, items.data(), 4 * items.size());
    if (!b->or_q.empty()) memcpy(h.data() + o_orq, b->or_q.data(), 4 * b->or_q.size());
    memcpy(h.data() + o_tb, tb.data(), 8ull * (nq + 1));
    // pinned mirrors: the upload source must stay valid until the copy runs
    uint8_t *hpin = nullptr;
    const uint64_t pin_bytes =
        align_up(o_up, 256) + align_up(sizeof(MStats) * std::max<uint32_t>(nq, 1), 256) + sizeof(MState) + 256;
    cudaError_t e = cudaSuccess;
    if (stage) {
        if (stage->cap < pin_bytes) {
            if (stage->p) cudaFreeHost(stage->p);
            stage->p = nullptr;
            stage->cap = 0;
            e = cudaMallocHost((void **)&stage->p, align_up(pin_bytes, 1 << 20));
            if (e == cudaSuccess) stage->cap = align_up(pin_bytes, 1 << 20);
        }
        hpin = stage->p;
    } else {
        e = cudaMallocHost((void **)&hpin, pin_bytes);
    }
    if (e != cudaSuccess) {
        if (native) dev_free_native(b->tables, s);
        else dev_free(b->tables, b->tables_bytes, s);
        delete b;
        return cuda_err(e, "multi-way pinned staging");
    }
    memcpy(hpin, h.data(), o_up);
    b->hpin = stage ? nullptr : hpin;
    b->h_stats = (MStats *)(hpin + align_up(o_up, 256));
    b->h_es = (MState *)((uint8_t *)b->h_stats + align_up(sizeof(MStats) * std::max<uint32_t>(nq, 1), 256));
    e = cudaMemcpyAsync(b->tables, hpin, o_up, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        if (!stage) cudaFreeHost(hpin);
        if (native) dev_free_native(b->tables, s);
        else dev_free(b->tables, b->tables_bytes, s);
        delete b;
        return cuda_err(e, "multi-way upload");
    }
    // the pinned block is released in multi_free, after the stream has run
    *out = b;
    *arena_bytes = b->arena_bytes;
    return RB_OK;
}

// CTAs of k_multi<W> resident per SM on the current device: found once per
// device from the occupancy calculator (after raising the kernel's dynamic
// shared-memory limit on that device); concurrent first calls store the same
// value
template <int W>
static int multi_ctas_per_sm() {
    constexpr int MAX_DEV = 256;
    static std::atomic<int> cache[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    int c = dev < MAX_DEV ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (c > 0) return c;
    const int smem = W * WARP_SMEM;
    cudaFuncSetAttribute(k_multi<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_multi<W>, W * 32, smem) != cudaSuccess || c < 1) {
        cudaGetLastError();
        c = 1;
    }
    if (dev < MAX_DEV) cache[dev].store(c, std::memory_order_relaxed);
    return c;
}

// k_multi is persistent: as many CTAs per SM as fit (16 warps per SM),
// capped by the batch's tiles
template <int W>
static void launch_multi_w(const MParams &P, cudaStream_t s) {
    const int smem = W * WARP_SMEM;
    const int ctas = multi_ctas_per_sm<W>();
    unsigned long long need = (P.n_tiles + W - 1) / W, cap = (unsigned long long)sm_count() * ctas;
    unsigned grid = (unsigned)std::max<unsigned long long>(1, std::min(need, cap));
    // chunks of consecutive tiles only when every warp has many tiles: a
    // small batch keeps one tile per warp at a time, for latency
    MParams Q = P;
    const unsigned long long per_warp = P.n_tiles / ((unsigned long long)grid * W);
    Q.chunk = per_warp >= 8ull * MCHUNK ? MCHUNK : 1;
    k_multi<W><<<grid, W * 32, smem, s>>>(Q);
}

rb_status multi_enqueue(MultiBatch *b, RbArena *arena, cudaStream_t s) {
    clear_stale_error();
    const uint32_t nq = (uint32_t)b->qd.size();
    MState &h = *b->h_es;
    memset(&h, 0, sizeof h);
    if (b->any_mat) {
        if (!arena || arena->bytes < b->arena_bytes) return set_err(RB_EINVAL, "multi-way arena too small");
        h.arena = (uint8_t *)arena->ptr;
        h.descs = (uint64_t *)arena->ptr;
        h.keys = (uint16_t *)((uint8_t *)arena->ptr + b->o_keys);
        h.words_off = b->o_words;
        h.words_cap = b->words_cap;
        h.bits_off = b->o_bits;
        h.bits_cap = b->bits_cap;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_es, b->h_es, sizeof(MState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nq) e = cudaMemsetAsync(b->d_stats, 0, sizeof(MStats) * nq, s);
    if (e == cudaSuccess && b->n_or) e = cudaMemsetAsync(b->d_pres, 0, 8192ull * b->n_or, s);
    if (e != cudaSuccess) return cuda_err(e, "multi-way enqueue");
    if (b->n_or) {
        const unsigned g1 = std::min<unsigned>(b->n_items, (unsigned)sm_count() * 16);
        k_presence<<<std::max(1u, g1), 256, 0, s>>>(b->d_pool, b->d_qs, b->d_members, b->d_items, b->n_items, b->d_pres);
        const unsigned g2 = std::min<unsigned>(b->n_or, (unsigned)sm_count() * 2);
        k_rank<<<std::max(1u, g2), 1024, 0, s>>>(b->d_qs, b->d_orq, b->n_or, b->d_pres, b->d_prefix, b->d_stats);
    }
    MParams P;
    P.pool = b->d_pool;
    P.qs = b->d_qs;
    P.members = b->d_members;
    P.moff = b->d_moff;
    P.tile_base = b->d_tb;
    P.pres = b->d_pres;
    P.prefix = b->d_prefix;
    P.stats = b->d_stats;
    P.es = b->d_es;
    P.n_tiles = b->total_tiles;
    P.n_q = nq;
    P.chunk = 1;
    const rb_schedule sc = current_schedule();
    if (b->total_tiles) {
        switch (sc.warps_per_cta) {
            case 2: launch_multi_w<2>(P, s); break;
            case 8: launch_multi_w<8>(P, s); break;
            default: launch_multi_w<4>(P, s); break;
        }
    }
    if (b->any_mat) {
        const unsigned g = std::max(1u, std::min<unsigned>(nq, (unsigned)sm_count() * 8));
        k_mcompact<<<g, 512, 0, s>>>(b->d_qs, nq, b->d_stats, b->d_es);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess && nq) e = cudaMemcpyAsync(b->h_stats, b->d_stats, sizeof(MStats) * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_es, b->d_es, sizeof(MState), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_err(e, "multi-way launch");
    return RB_OK;
}

rb_status multi_finish(MultiBatch *b, RbArena *arena, rb_t **outs, uint64_t *cards) {
    if (b->h_es->status & 1u) return set_err(RB_ENOMEM, "multi-way: result bound exceeded (internal error)");
    for (size_t q = 0; q < b->qd.size(); q++) {
        const MultiDev &d = b->qd[q];
        const MStats &S = b->h_stats[q];
        if (cards) cards[q] = S.card;
        if (!outs) continue;
        if (d.count_only) { outs[q] = nullptr; continue; }
        rb *h = handle_new();
        h->n = S.n_out;
        h->card = S.card;
        h->word_bytes = S.words;
        h->n_bitsets = S.nbits;
        h->base = (uint8_t *)arena->ptr;
        h->descs = (uint64_t *)arena->ptr + d.slot_base;
        h->keys = (uint16_t *)((uint8_t *)arena->ptr + b->o_keys) + d.slot_base;
        h->arena = arena;
        arena_ref(arena);
        outs[q] = h;
    }
    return RB_OK;
}

void multi_free(MultiBatch *b, cudaStream_t s) {
    if (!b) return;
    if (b->tables) {
        if (b->native) dev_free_native(b->tables, s);
        else dev_free(b->tables, b->tables_bytes, s);
    }
    if (b->hpin) cudaFreeHost(b->hpin);
    delete b;
}

}  // namespace rbi

extern "C" rb_status rb_multi_op(rb_op op, const rb_t *const *in, uint32_t k, rb_t **out, uint64_t *card,
                                 void *stream) {
    if (out) *out = nullptr;
    if (op != RB_AND && op != RB_OR) return set_err(RB_EINVAL, "rb_multi_op: op must be RB_AND or RB_OR");
    if (k && !in) return set_err(RB_EINVAL, "rb_multi_op: NULL inputs");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<BmView> hv(k);
    for (uint32_t i = 0; i < k; i++) {
        if (!in[i]) return set_err(RB_EINVAL, "rb_multi_op: in[%u] is NULL", i);
        hv[i] = view_of(in[i]);
    }
    BmView *dv = (BmView *)dev_alloc(sizeof(BmView) * std::max<uint32_t>(k, 1), s);
    if (!dv) return RB_ENOMEM;
    cudaError_t e = k ? cudaMemcpyAsync(dv, hv.data(), sizeof(BmView) * k, cudaMemcpyHostToDevice, s) : cudaSuccess;
    if (e != cudaSuccess) { dev_free(dv, sizeof(BmView) * std::max<uint32_t>(k, 1), s); return cuda_err(e, "rb_multi_op"); }
    MultiQuery mq;
    mq.op = (uint32_t)op;
    mq.count_only = out ? 0 : 1;
    for (uint32_t i = 0; i < k; i++) mq.members.push_back(i);
    std::vector<MultiQuery> qs(1, mq);
    MultiBatch *b = nullptr;
    uint64_t ab = 0;
    rb_status st = multi_prepare(in, dv, k, qs, s, &b, &ab);
    RbArena *a = nullptr;
    if (st == RB_OK && ab) {
        a = arena_new(ab, s);
        if (!a) st = RB_ENOMEM;
    }
    if (st == RB_OK) st = multi_enqueue(b, a, s);
    if (st == RB_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_err(e, "rb_multi_op");
    }
    uint64_t c = 0;
    if (st == RB_OK) st = multi_finish(b, a, out ? out : nullptr, &c);
    if (st == RB_OK && card) *card = c;
    if (b) multi_free(b, s);
    arena_unref(a);
    dev_free(dv, sizeof(BmView) * std::max<uint32_t>(k, 1), s);
    return st;
}
