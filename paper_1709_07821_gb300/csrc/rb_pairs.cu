// rb_pairs.cu - pairwise operations: key merge, container-pair kernels,
// canonical compaction, batches, plans (CUDA graphs) and the autotuner.
//
// Work decomposition.  Every query (a op b) owns a range of "slots"; a slot
// is one key of one input and becomes at most one output container:
//   AND (and every count-only query): the keys of the input with fewer keys;
//   ANDNOT: the keys of a;  OR / XOR: the keys of a, then the keys of b.
// A slot finds its partner by binary search in the other key array (the key
// merge of Sec. 5's profiles, done per slot), so a key present in both
// inputs becomes one container pair.  Its output position keeps the key
// order of the result: the slot index for AND/ANDNOT, and for OR/XOR the
// merge-path position in the multiset of both key lists (a's key first on a
// tie; b's copy of a shared key only marks its position empty).  Every
// position of a query's slot range is written exactly once, so the
// compaction pass only has to drop empty results.
// Slots are cut into tiles of 32; warps of a persistent kernel steal tiles
// from one atomic counter.  In a tile each lane resolves its container pair;
// small pairs (few values or runs on both sides) are merged by the lane alone
// with an interval sweep, large ones by the whole warp through 8 KB shared
// tiles (bitset operands are read straight from global memory).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rb_device.cuh"

using namespace rbi;
using namespace rbd;

namespace {

constexpr uint32_t F_COUNT = 1;
enum : uint32_t { K_NONE = 0, K_EMPTY = 1, K_PAIR = 2, K_COPY_A = 3, K_COPY_B = 4 };

struct PairDev {
    uint32_t a, b, op, flags;
    uint32_t n_slots, pad;
    unsigned long long slot_base;
};

struct PairStats {
    unsigned long long card;      // output cardinality (count-only: |a n b|)
    unsigned long long words;     // word-region bytes of the output
    unsigned long long in_bytes;  // algorithmic input bytes read
    unsigned int n_out, m, nbits, pad;
};

struct ExecState {
    uint8_t *arena;
    uint16_t *keys;
    uint64_t *descs;
    unsigned long long words_off, words_cap, bits_off, bits_cap;
    unsigned long long words_used, bits_used, work;
    unsigned int status, pad;
};

struct PairParams {
    const BmView *pool;
    const PairDev *pairs;
    const unsigned long long *tile_base;
    PairStats *stats;
    ExecState *es;
    unsigned long long n_tiles;
    uint32_t n_pairs;
    uint32_t small_iv;
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

// ------------------------------------------------------------ warp paths

__device__ uint64_t warp_copy(ExecState *es, const CRef &x, uint32_t lane) {
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
    const uint32_t *S = reinterpret_cast<const uint32_t *>(x.p);
    uint32_t *D = reinterpret_cast<uint32_t *>(es->arena + off);
    for (uint32_t i = lane; i < bytes / 4; i += 32) D[i] = __ldg(S + i);
    return mk_desc(x.card, x.type, x.type == T_RUN ? x.runs : 0, off);
}

// a op b for one container pair by the whole warp; returns the output
// descriptor (DESC_EMPTY for an empty result or a failed allocation)
__device__ uint64_t warp_pair(ExecState *es, uint32_t op, const CRef &a, const CRef &b, uint64_t *T0, uint64_t *T1,
                              uint32_t lane) {
    const bool a_arr = a.type == T_ARRAY, b_arr = b.type == T_ARRAY;
    if ((op == OP_AND && (a_arr || b_arr)) || (op == OP_ANDNOT && a_arr)) {
        // the result is a subset of an array: test each of its values
        // against the other container (Sec. 3.2 bit tests)
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
        const uint64_t off = alloc_words_warp(es, word_alloc_bytes(ty, c, r), lane);
        if (off == ALLOC_FAIL) return DESC_EMPTY;
        if (ty == T_ARRAY) l_emit_array(L, c, reinterpret_cast<uint16_t *>(es->arena + off), lane);
        else l_emit_runs(L, c, r, reinterpret_cast<uint16_t *>(T0), reinterpret_cast<uint32_t *>(es->arena + off), lane);
        return mk_desc(c, ty, ty == T_RUN ? r : 0, off);
    }
    // general case: both operands as 2^16-bit words, combined word by word
    const uint64_t *sa, *sb;
    if (a.type == T_BITSET) sa = reinterpret_cast<const uint64_t *>(a.p);
    else { t_decode(T0, a, lane); sa = T0; }
    if (b.type == T_BITSET) sb = reinterpret_cast<const uint64_t *>(b.p);
    else { t_decode(T1, b, lane); sb = T1; }
    uint32_t c, r;
    t_combine<true>(T0, sa, sb, op, c, r, lane);
    __syncwarp();
    if (c == 0) return DESC_EMPTY;
    const uint32_t ty = canon_type(c, r);
    uint64_t off;
    if (ty == T_BITSET) {
        off = alloc_bitset_warp(es, lane);
        if (off == ALLOC_FAIL) return DESC_EMPTY;
        t_emit_bitset(T0, reinterpret_cast<uint64_t *>(es->arena + off), lane);
    } else {
        off = alloc_words_warp(es, word_alloc_bytes(ty, c, r), lane);
        if (off == ALLOC_FAIL) return DESC_EMPTY;
        if (ty == T_ARRAY) {
            t_emit_array(T0, reinterpret_cast<uint16_t *>(es->arena + off), lane);
        } else {
            uint16_t *S = reinterpret_cast<uint16_t *>(T1);
            t_emit_runs(T0, S, S + 2048, reinterpret_cast<uint32_t *>(es->arena + off), r, lane);
        }
    }
    return mk_desc(c, ty, ty == T_RUN ? r : 0, off);
}

// |a n b| for one container pair by the whole warp
__device__ uint32_t warp_count_and(const CRef &a, const CRef &b, uint64_t *T0, uint64_t *T1, uint32_t lane) {
    const bool a_arr = a.type == T_ARRAY, b_arr = b.type == T_ARRAY;
    uint32_t c;
    if (a_arr || b_arr) {
        const CRef *X = (a_arr && b_arr) ? (a.card <= b.card ? &a : &b) : (a_arr ? &a : &b);
        const CRef *O = (X == &a) ? &b : &a;
        const uint64_t *ow;
        if (O->type == T_BITSET) ow = reinterpret_cast<const uint64_t *>(O->p);
        else { t_decode(T0, *O, lane); ow = T0; }
        c = probe_list<false>(reinterpret_cast<const uint16_t *>(X->p), X->card, ow, 1, nullptr, lane);
    } else {
        const uint64_t *sa, *sb;
        if (a.type == T_BITSET) sa = reinterpret_cast<const uint64_t *>(a.p);
        else { t_decode(T0, a, lane); sa = T0; }
        if (b.type == T_BITSET) sb = reinterpret_cast<const uint64_t *>(b.p);
        else { t_decode(T1, b, lane); sb = T1; }
        uint32_t r;
        t_combine<false>(nullptr, sa, sb, OP_AND, c, r, lane);
    }
    __syncwarp();
    return c;
}

// ------------------------------------------------------------ one tile

__device__ void pair_tile(const PairParams &P, unsigned long long t, uint64_t *T0, uint64_t *T1, uint32_t lane) {
    // the query owning tile t: largest p with tile_base[p] <= t
    uint32_t lo = 0, hi = P.n_pairs;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (P.tile_base[mid] <= t) lo = mid;
        else hi = mid;
    }
    const uint32_t p = lo;
    const PairDev pd = P.pairs[p];
    const BmView A = P.pool[pd.a], B = P.pool[pd.b];
    ExecState *es = P.es;
    const uint32_t op = pd.op;
    const bool count_only = (pd.flags & F_COUNT) != 0;
    const uint32_t slot = (uint32_t)(t - P.tile_base[p]) * 32u + lane;

    // ---- key merge for this lane's slot
    uint32_t kind = K_NONE, key = 0, pos = 0, ia = 0, ib = 0, matchedA = 0;
    if (slot < pd.n_slots) {
        if (count_only || op == OP_AND) {
            const bool drvA = A.n <= B.n;
            const uint16_t *dk = drvA ? A.keys : B.keys;
            const uint16_t *ok = drvA ? B.keys : A.keys;
            const uint32_t on = drvA ? B.n : A.n;
            key = __ldg(dk + slot);
            const uint32_t j = lower_bound16(ok, on, key);
            pos = slot;
            if (j < on && __ldg(ok + j) == key) {
                kind = K_PAIR;
                ia = drvA ? slot : j;
                ib = drvA ? j : slot;
            } else {
                kind = K_EMPTY;
            }
        } else if (op == OP_ANDNOT) {
            key = __ldg(A.keys + slot);
            const uint32_t j = lower_bound16(B.keys, B.n, key);
            pos = slot;
            ia = slot;
            if (j < B.n && __ldg(B.keys + j) == key) { kind = K_PAIR; ib = j; }
            else kind = K_COPY_A;
        } else if (slot < A.n) {
            key = __ldg(A.keys + slot);
            const uint32_t j = lower_bound16(B.keys, B.n, key);
            pos = slot + j;
            ia = slot;
            if (j < B.n && __ldg(B.keys + j) == key) { kind = K_PAIR; ib = j; matchedA = 1; }
            else kind = K_COPY_A;
        } else {
            // merge-path position over the multiset of both key lists (a's
            // key first on a tie): a key b shares with a sits right after a's
            // and only marks its position empty
            const uint32_t jb = slot - A.n;
            key = __ldg(B.keys + jb);
            const uint32_t i = lower_bound16(A.keys, A.n, key);
            if (i < A.n && __ldg(A.keys + i) == key) { kind = K_EMPTY; pos = jb + i + 1; }
            else { kind = K_COPY_B; ib = jb; pos = jb + i; }
        }
    }
    const uint64_t da = (kind == K_PAIR || kind == K_COPY_A) ? __ldg(A.descs + ia) : 0ull;
    const uint64_t db = (kind == K_PAIR || kind == K_COPY_B) ? __ldg(B.descs + ib) : 0ull;
    unsigned long long inb = 0;
    if (kind == K_PAIR) inb = in_payload_bytes(da) + in_payload_bytes(db) + 18;
    else if (kind == K_COPY_A) inb = in_payload_bytes(da) + 10;
    else if (kind == K_COPY_B) inb = in_payload_bytes(db) + 10;
    else if (kind == K_EMPTY) inb = 10;

    if (count_only) {
        // Sec. 5 "Fast counts": only |a n b| is computed
        uint32_t cnt = 0;
        bool large = false;
        if (kind == K_PAIR) {
            if (n_intervals(da) + n_intervals(db) <= P.small_iv) {
                uint32_t c, r;
                const CRef ca = cref(A.base, da), cb = cref(B.base, db);
                lane_sweep<false>(OP_AND, iv_src(ca), iv_src(cb), c, r, 0, nullptr);
                cnt = c;
            } else {
                large = true;
            }
        }
        unsigned long long wc = 0;
        uint32_t lm = __ballot_sync(FULL, large);
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const uint64_t xa = __shfl_sync(FULL, da, src), xb = __shfl_sync(FULL, db, src);
            wc += warp_count_and(cref(A.base, xa), cref(B.base, xb), T0, T1, lane);
        }
        const unsigned long long tot = warp_sum64(cnt) + wc, ib_tot = warp_sum64(inb);
        if (lane == 0) {
            if (tot) atomicAdd(&P.stats[p].card, tot);
            atomicAdd(&P.stats[p].in_bytes, ib_tot);
        }
        return;
    }

    // ---- materialise
    bool small = false, large = false;
    if (kind == K_PAIR) {
        if (n_intervals(da) + n_intervals(db) <= P.small_iv) small = true;
        else large = true;
    } else if (kind == K_COPY_A || kind == K_COPY_B) {
        if (n_intervals(kind == K_COPY_A ? da : db) <= P.small_iv) small = true;
        else large = true;
    }
    uint32_t lc = 0, lr = 0, lt = 0, lbytes = 0;
    CRef ca, cb;
    ca.p = nullptr;
    cb.p = nullptr;
    if (small) {
        if (kind == K_PAIR) {
            ca = cref(A.base, da);
            cb = cref(B.base, db);
            lane_sweep<false>(op, iv_src(ca), iv_src(cb), lc, lr, 0, nullptr);
            if (lc) {
                lt = canon_type(lc, lr);
                lbytes = word_alloc_bytes(lt, lc, lr);
            }
        } else {
            const uint64_t dx = kind == K_COPY_A ? da : db;
            ca = cref(kind == K_COPY_A ? A.base : B.base, dx);
            lc = ca.card;
            lr = ca.runs;
            lt = ca.type;
            lbytes = word_alloc_bytes(lt, lc, lr);
        }
    }
    // one atomic per warp for all lane-sized outputs
    const uint32_t incl = warp_incl(lbytes, lane);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    unsigned long long wbase = 0;
    bool ok = true;
    if (total) {
        if (lane == 31) wbase = atomicAdd(&es->words_used, (unsigned long long)total);
        wbase = __shfl_sync(FULL, wbase, 31);
        ok = wbase + total <= es->words_cap;
        if (!ok && lane == 0) atomicOr(&es->status, 1u);
    }
    uint16_t *OKEY = es->keys + pd.slot_base;
    uint64_t *ODESC = es->descs + pd.slot_base;
    unsigned long long card_acc = 0, words_acc = 0;
    uint32_t bits_acc = 0;
    if (small) {
        uint64_t desc = DESC_EMPTY;
        if (lc && ok) {
            const uint64_t off = es->words_off + wbase + incl - lbytes;
            uint8_t *dst = es->arena + off;
            if (kind == K_PAIR) {
                uint32_t c2, r2;
                lane_sweep<true>(op, iv_src(ca), iv_src(cb), c2, r2, lt, dst);
            } else {
                const uint32_t *S = reinterpret_cast<const uint32_t *>(ca.p);
                uint32_t *D = reinterpret_cast<uint32_t *>(dst);
                for (uint32_t i = 0; i < lbytes / 4; i++) D[i] = __ldg(S + i);
            }
            desc = mk_desc(lc, lt, lt == T_RUN ? lr : 0, off);
            card_acc += lc;
            words_acc += lbytes;
        }
        ODESC[pos] = desc;
        OKEY[pos] = (uint16_t)key;
    } else if (kind == K_EMPTY) {
        ODESC[pos] = DESC_EMPTY;
        OKEY[pos] = (uint16_t)key;
    }
    uint32_t lm = __ballot_sync(FULL, large);
    while (lm) {
        const int src = __ffs(lm) - 1;
        lm &= lm - 1;
        const uint32_t k_s = __shfl_sync(FULL, kind, src);
        const uint32_t pos_s = __shfl_sync(FULL, pos, src);
        const uint32_t key_s = __shfl_sync(FULL, key, src);
        const uint64_t da_s = __shfl_sync(FULL, da, src), db_s = __shfl_sync(FULL, db, src);
        uint64_t desc;
        if (k_s == K_PAIR) desc = warp_pair(es, op, cref(A.base, da_s), cref(B.base, db_s), T0, T1, lane);
        else desc = warp_copy(es, k_s == K_COPY_A ? cref(A.base, da_s) : cref(B.base, db_s), lane);
        if (lane == 0) {
            ODESC[pos_s] = desc;
            OKEY[pos_s] = (uint16_t)key_s;
            if (desc != DESC_EMPTY) {
                card_acc += d_card(desc);
                if (d_type(desc) == T_BITSET) bits_acc++;
                else words_acc += word_alloc_bytes(d_type(desc), d_card(desc), d_runs(desc));
            }
        }
        __syncwarp();
    }
    const unsigned long long cs = warp_sum64(card_acc), ws = warp_sum64(words_acc), is = warp_sum64(inb);
    const uint32_t bs = warp_sum(bits_acc), ms = __popc(__ballot_sync(FULL, matchedA));
    if (lane == 0) {
        PairStats *S = P.stats + p;
        if (cs) atomicAdd(&S->card, cs);
        if (ws) atomicAdd(&S->words, ws);
        if (is) atomicAdd(&S->in_bytes, is);
        if (bs) atomicAdd(&S->nbits, bs);
        if (ms) atomicAdd(&S->m, ms);
    }
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) k_pairs(PairParams P) {
    extern __shared__ __align__(16) uint64_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *T0 = smem + (size_t)warp * 2048;
    uint64_t *T1 = T0 + 1024;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&P.es->work, 1ull);
        t = __shfl_sync(FULL, t, 0);
        if (t >= P.n_tiles) break;
        pair_tile(P, t, T0, T1, lane);
    }
}

// drop empty results: in-place stream compaction of each query's slot range
// (positions are already in key order), one block per query
__global__ void __launch_bounds__(512) k_compact(const PairDev *pairs, uint32_t n_pairs, PairStats *stats,
                                                 const ExecState *es) {
    __shared__ uint32_t s_w[16];
    __shared__ uint32_t s_tot;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (uint32_t p = blockIdx.x; p < n_pairs; p += gridDim.x) {
        const PairDev pd = pairs[p];
        if (pd.flags & F_COUNT) continue;
        const uint32_t n = pd.n_slots;   // every position of the slot range is written once
        uint64_t *D = es->descs + pd.slot_base;
        uint16_t *K = es->keys + pd.slot_base;
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

template <int W>
void launch_pairs_w(const PairParams &P, int ctas_per_sm, cudaStream_t s) {
    static bool attr = false;
    const int smem = W * 16384;
    if (!attr) {
        cudaFuncSetAttribute(k_pairs<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    unsigned long long need = (P.n_tiles + W - 1) / W;
    unsigned long long cap = (unsigned long long)sm_count() * (unsigned long long)ctas_per_sm;
    unsigned grid = (unsigned)std::max<unsigned long long>(1, std::min(need, cap));
    k_pairs<W><<<grid, W * 32, smem, s>>>(P);
}

void launch_pairs(const PairParams &P, const rb_schedule &sc, cudaStream_t s) {
    switch (sc.warps_per_cta) {
        case 2: launch_pairs_w<2>(P, sc.ctas_per_sm, s); break;
        case 8: launch_pairs_w<8>(P, sc.ctas_per_sm, s); break;
        default: launch_pairs_w<4>(P, sc.ctas_per_sm, s); break;
    }
}

}  // namespace

struct rb_plan {
    std::vector<const rb *> pool;
    std::vector<rb_query> q;
    std::vector<PairDev> pairs;
    uint64_t total_slots = 0, total_tiles = 0;
    uint64_t words_cap = 0, bits_cap = 0;   // arena sizes for the next run
    bool exact = false;                     // caps measured by a previous run
    bool any_mat = false;
    uint8_t *tables = nullptr;
    uint64_t tables_bytes = 0;
    BmView *d_pool = nullptr;
    PairDev *d_pairs = nullptr;
    unsigned long long *d_tile_base = nullptr;
    PairStats *d_stats = nullptr;
    ExecState *d_es = nullptr;
    PairStats *h_stats = nullptr;
    ExecState *h_es = nullptr;
    cudaStream_t ps = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_in = nullptr;
    cudaGraphExec_t gexec = nullptr;
    rb_schedule gsched = {0, 0, 0, 0};
    double last_ms = 0;
    uint64_t last_alg = 0, last_out = 0;
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
    if (p->ev_in) cudaEventDestroy(p->ev_in);
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
    uint64_t slots = 0, tiles = 0, ew = 0, eb = 0, bw = 0, bb = 0;
    for (uint64_t i = 0; i < nq; i++) {
        const rb_query &x = q[i];
        if (x.op > 3 || x.a >= pool_n || x.b >= pool_n) {
            plan_destroy(p);
            return set_err(RB_EINVAL, "batch: query %llu has op %u, a %u, b %u (pool of %u)",
                           (unsigned long long)i, x.op, x.a, x.b, pool_n);
        }
        const rb *A = pool[x.a], *B = pool[x.b];
        PairDev &d = p->pairs[i];
        d.a = x.a;
        d.b = x.b;
        d.op = x.op;
        d.flags = (x.flags & RB_Q_COUNT_ONLY) ? F_COUNT : 0;
        uint64_t ns;
        if ((d.flags & F_COUNT) || x.op == OP_AND) ns = std::min(A->n, B->n);
        else if (x.op == OP_ANDNOT) ns = A->n;
        else ns = (uint64_t)A->n + B->n;
        d.n_slots = (uint32_t)ns;
        d.pad = 0;
        d.slot_base = (d.flags & F_COUNT) ? 0 : slots;
        if (!(d.flags & F_COUNT)) {
            slots += ns;
            p->any_mat = true;
            uint64_t w1, b1;
            query_bounds(A, B, x.op, w1, b1);
            bw += w1;
            bb += b1;
            if (x.op == OP_AND) {
                ew += std::min(A->word_bytes, B->word_bytes);
                eb += 8192ull * std::min(A->n_bitsets, B->n_bitsets);
            } else if (x.op == OP_ANDNOT) {
                ew += A->word_bytes;
                eb += 8192ull * A->n_bitsets;
            } else {
                ew += A->word_bytes + B->word_bytes;
                eb += 8192ull * ((uint64_t)A->n_bitsets + B->n_bitsets);
            }
        }
        tb[i] = tiles;
        tiles += (ns + 31) / 32;
    }
    tb[nq] = tiles;
    p->total_slots = slots;
    p->total_tiles = tiles;
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
    const uint64_t o_tb = align_up(o_pairs + sizeof(PairDev) * nq, 256);
    const uint64_t o_stats = align_up(o_tb + 8ull * (nq + 1), 256);
    const uint64_t o_es = align_up(o_stats + sizeof(PairStats) * nq, 256);
    p->tables_bytes = o_es + 256;
    p->tables = (uint8_t *)dev_alloc(p->tables_bytes, s);
    if (!p->tables) { plan_destroy(p); return RB_ENOMEM; }
    p->d_pool = (BmView *)(p->tables + o_pool);
    p->d_pairs = (PairDev *)(p->tables + o_pairs);
    p->d_tile_base = (unsigned long long *)(p->tables + o_tb);
    p->d_stats = (PairStats *)(p->tables + o_stats);
    p->d_es = (ExecState *)(p->tables + o_es);
    // host staging: pool views, then everything goes up in one copy
    std::vector<uint8_t> hbuf(o_stats);
    BmView *hv = (BmView *)(hbuf.data() + o_pool);
    for (uint32_t i = 0; i < pool_n; i++) hv[i] = view_of(pool[i]);
    if (nq) memcpy(hbuf.data() + o_pairs, p->pairs.data(), sizeof(PairDev) * nq);
    memcpy(hbuf.data() + o_tb, tb.data(), 8ull * (nq + 1));
    cudaError_t e = cudaMallocHost((void **)&p->h_stats, sizeof(PairStats) * std::max<uint64_t>(nq, 1));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&p->h_es, sizeof(ExecState));
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->tables, hbuf.data(), o_stats, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&p->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        plan_destroy(p);
        return cuda_err(e, "plan setup");
    }
    *out = p;
    return RB_OK;
}

// the launch sequence of one run, enqueued on stream s
// capture: the events become external event-record nodes of the graph, so
// the kernel's time can still be read after a replay
cudaError_t enqueue_run(rb_plan *p, const rb_schedule &sc, cudaStream_t s, bool capture) {
    const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
    const uint64_t nq = p->q.size();
    cudaError_t e = cudaMemcpyAsync(p->d_es, p->h_es, sizeof(ExecState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nq) e = cudaMemsetAsync(p->d_stats, 0, sizeof(PairStats) * nq, s);
    if (e != cudaSuccess) return e;
    PairParams P;
    P.pool = p->d_pool;
    P.pairs = p->d_pairs;
    P.tile_base = p->d_tile_base;
    P.stats = p->d_stats;
    P.es = p->d_es;
    P.n_tiles = p->total_tiles;
    P.n_pairs = (uint32_t)nq;
    P.small_iv = sc.small_intervals;
    if ((e = cudaEventRecordWithFlags(p->ev0, s, evf)) != cudaSuccess) return e;
    if (p->total_tiles) launch_pairs(P, sc, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(p->ev1, s, evf)) != cudaSuccess) return e;
    if (p->any_mat) {
        unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(nq, (uint64_t)sm_count() * 8));
        k_compact<<<grid, 512, 0, s>>>(p->d_pairs, (uint32_t)nq, p->d_stats, p->d_es);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (nq) e = cudaMemcpyAsync(p->h_stats, p->d_stats, sizeof(PairStats) * nq, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_es, p->d_es, sizeof(ExecState), cudaMemcpyDeviceToHost, s);
    return e;
}

// one run with the plan's current caps; on success *arena holds the results
// (NULL when every query is count-only); *overflow tells the caller to retry
rb_status run_once(rb_plan *p, cudaStream_t s, bool graph, RbArena **arena, bool *overflow) {
    *arena = nullptr;
    *overflow = false;
    const rb_schedule sc = current_schedule();
    const uint64_t T = p->total_slots;
    const uint64_t o_keys = align_up(8 * T, 256);
    const uint64_t o_words = align_up(o_keys + 2 * T, 256);
    const uint64_t o_bits = align_up(o_words + p->words_cap, 256);
    const uint64_t bytes = o_bits + p->bits_cap;
    if (p->any_mat && bytes >= MAX_OFFSET)
        return set_err(RB_ERANGE, "batch results need %llu bytes, above the 128 GiB descriptor reach; split the batch",
                       (unsigned long long)bytes);
    RbArena *a = nullptr;
    if (p->any_mat) {
        a = arena_new(bytes, s);
        if (!a) return RB_ENOMEM;
    }
    ExecState &h = *p->h_es;
    memset(&h, 0, sizeof h);
    if (a) {
        h.arena = (uint8_t *)a->ptr;
        h.descs = (uint64_t *)a->ptr;
        h.keys = (uint16_t *)((uint8_t *)a->ptr + o_keys);
        h.words_off = o_words;
        h.words_cap = p->words_cap;
        h.bits_off = o_bits;
        h.bits_cap = p->bits_cap;
    }
    cudaError_t e = cudaSuccess;
    if (graph) {
        if (!p->ps) e = cudaStreamCreateWithFlags(&p->ps, cudaStreamNonBlocking);
        if (e == cudaSuccess && p->gexec &&
            memcmp(&p->gsched, &sc, sizeof sc) != 0) {
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
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->ps);
    } else {
        e = enqueue_run(p, sc, s, false);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        arena_unref(a);
        return cuda_err(e, "batch run");
    }
    float ms = 0.f;
    if (p->total_tiles && cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess) p->last_ms = ms;
    else p->last_ms = 0;
    cudaGetLastError();
    if (h.status & 1u) {
        *overflow = true;
        p->words_cap = h.words_used;
        p->bits_cap = h.bits_used;
        arena_unref(a);
        return RB_OK;
    }
    if (!p->exact) {
        p->words_cap = h.words_used;
        p->bits_cap = h.bits_used;
        p->exact = true;
    }
    *arena = a;
    return RB_OK;
}

rb_status plan_execute(rb_plan *p, rb_t **outs, uint64_t *counts, cudaStream_t s, bool graph) {
    clear_stale_error();
    RbArena *a = nullptr;
    bool overflow = false;
    rb_status st = RB_OK;
    for (int attempt = 0; attempt < 3; attempt++) {
        st = run_once(p, s, graph && attempt > 0 ? false : graph, &a, &overflow);
        if (st != RB_OK) return st;
        if (!overflow) break;
    }
    if (overflow) return set_err(RB_ENOMEM, "batch: output arena overflow persisted");
    const uint64_t nq = p->q.size();
    const uint64_t T = p->total_slots;
    const uint64_t o_keys = align_up(8 * T, 256);
    uint64_t alg = 0, outb = 0;
    for (uint64_t i = 0; i < nq; i++) {
        const PairDev &d = p->pairs[i];
        const PairStats &S = p->h_stats[i];
        const rb *A = p->pool[d.a], *B = p->pool[d.b];
        alg += S.in_bytes;
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
            alg += 8;
            if (outs) outs[i] = nullptr;
            continue;
        }
        const uint64_t ob = S.words + 8192ull * S.nbits + 10ull * S.n_out;
        alg += ob;
        outb += ob;
        if (counts) counts[i] = S.card;
        if (outs) {
            rb *h = handle_new();
            h->n = S.n_out;
            h->card = S.card;
            h->word_bytes = S.words;
            h->n_bitsets = S.nbits;
            h->base = (uint8_t *)a->ptr;
            h->descs = (uint64_t *)a->ptr + d.slot_base;
            h->keys = (uint16_t *)((uint8_t *)a->ptr + o_keys) + d.slot_base;
            h->arena = a;
            arena_ref(a);
            outs[i] = h;
        }
    }
    p->last_alg = alg;
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
    if (outs)
        for (uint64_t i = 0; i < p->q.size(); i++) outs[i] = nullptr;
    if (p->any_mat && !outs) return set_err(RB_EINVAL, "rb_plan_run: outs is NULL but the plan materialises");
    // the first run sizes the arena exactly; later runs replay a CUDA graph
    return plan_execute(p, outs, counts, (cudaStream_t)stream, p->exact);
}

rb_status rb_plan_stats(const rb_plan_t *p, double *kernel_ms, uint64_t *alg_bytes, uint64_t *out_bytes) {
    if (!p) return set_err(RB_EINVAL, "rb_plan_stats: NULL plan");
    if (kernel_ms) *kernel_ms = p->last_ms;
    if (alg_bytes) *alg_bytes = p->last_alg;
    if (out_bytes) *out_bytes = p->last_out;
    return RB_OK;
}

void rb_plan_free(rb_plan_t *p) { plan_destroy(p); }

rb_status rb_autotune(rb_plan_t *p, uint32_t reps, void *stream, rb_schedule *best, double *best_ms) {
    if (!p) return set_err(RB_EINVAL, "rb_autotune: NULL plan");
    if (reps == 0) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    const rb_schedule saved = current_schedule();
    static const uint32_t shapes[][2] = {{2, 6}, {4, 3}, {8, 1}};
    static const uint32_t smalls[] = {8, 32, 128, 512};
    rb_schedule win = saved;
    double win_ms = 1e30;
    std::vector<rb_t *> outs(p->q.size(), nullptr);
    for (auto &sh : shapes) {
        for (uint32_t sm : smalls) {
            rb_schedule c = {sh[0], sh[1], sm, 0};
            if (rb_set_schedule(&c) != RB_OK) continue;
            double tot = 0;
            bool ok = true;
            for (uint32_t r = 0; r < reps + 1 && ok; r++) {
                rb_status st = plan_execute(p, outs.data(), nullptr, s, false);
                for (auto &h : outs) { rb_free(h); h = nullptr; }
                if (st != RB_OK) ok = false;
                else if (r > 0) tot += p->last_ms;   // first run is a warm-up
            }
            if (ok && tot / reps < win_ms) {
                win_ms = tot / reps;
                win = c;
            }
        }
    }
    rb_set_schedule(win_ms < 1e30 ? &win : &saved);
    if (best) *best = current_schedule();
    if (best_ms) *best_ms = win_ms;
    return win_ms < 1e30 ? RB_OK : set_err(RB_ECUDA, "rb_autotune: no schedule ran");
}

}  // extern "C"
