// rb_accum.cu - in-place accumulation: acc = acc op B over a stream of
// bitmaps, without allocating per call.
//
// Sec. 5 "Wide unions" computes the union of many bitmaps with a function
// that works partly in place, and Sec. 2.2 describes lazy operations that do
// not maintain the cardinality of intermediate results.  The accumulator
// keeps one 8 KB bitset tile per key present (a key -> tile map of 65536
// entries and a tile pool reserved at creation), updates the tiles in place
// on every add, and computes cardinalities, run counts and canonical
// container types only once, when the result is requested.
//
// OR add: one warp per container of B.  A key seen for the first time takes
// the next free tile (zeroed by its warp); a bitset is OR-ed word by word, an
// array sets its values' bits with atomic ORs and a run container sets its
// ranges (whole words by stores, the partial words at its ends by atomic
// ORs), so only the words the container touches are written.
// AND add: the first add fills the accumulator as OR does; later adds visit
// every key present, drop the keys B lacks and AND the tile with B's
// container (decoded into a shared-memory tile unless it is a bitset).
#include <cstring>
#include <vector>

#include "rb_device.cuh"

using namespace rbi;
using namespace rbd;

namespace {

constexpr uint32_t NO_TILE = 0xFFFFFFFFu;
constexpr uint32_t KEYS = 65536;

struct AccState {
    unsigned int used;     // tiles handed out
    unsigned int status;   // bit 0: the tile pool ran out
    unsigned int n_keys, n_bits;              // result: containers, bitset containers
    unsigned long long words, card;           // result: word-region bytes, cardinality
};

// per key of the result (k_acc_count): packed c - 1 (16 b), type (2 b),
// runs (11 b); ~0 when absent
__device__ __forceinline__ uint64_t pack_info(uint32_t c, uint32_t t, uint32_t r) {
    return (uint64_t)(c - 1) | ((uint64_t)t << 16) | ((uint64_t)r << 18);
}

__global__ void k_acc_or(uint32_t *map, uint64_t *tiles, AccState *st, uint32_t max_tiles, BmView B) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < B.n; i += warps) {
        const uint32_t key = __ldg(B.keys + i);
        uint32_t idx = 0;
        bool fresh = false;
        if (lane == 0) {
            idx = map[key];
            if (idx == NO_TILE) {
                idx = atomicAdd(&st->used, 1u);
                if (idx >= max_tiles) {
                    atomicOr(&st->status, 1u);
                    idx = NO_TILE;
                } else {
                    map[key] = idx;
                    fresh = true;
                }
            }
        }
        idx = __shfl_sync(FULL, idx, 0);
        fresh = __shfl_sync(FULL, fresh, 0);
        if (idx == NO_TILE) continue;
        uint64_t *T = tiles + (size_t)idx * 1024;
        const CRef x = cref(B.base, __ldg(B.descs + i));
        ulonglong2 *T2 = reinterpret_cast<ulonglong2 *>(T);
        if (x.type == T_BITSET) {
            const ulonglong2 *S = reinterpret_cast<const ulonglong2 *>(x.p);
#pragma unroll 4
            for (int k = 0; k < 16; k++) {
                const ulonglong2 s = __ldg(S + 32 * k + lane);
                if (fresh) {
                    T2[32 * k + lane] = s;
                } else {
                    const ulonglong2 t = T2[32 * k + lane];
                    T2[32 * k + lane] = make_ulonglong2(t.x | s.x, t.y | s.y);
                }
            }
            continue;
        }
        if (fresh) {
#pragma unroll 4
            for (int k = 0; k < 16; k++) T2[32 * k + lane] = make_ulonglong2(0ull, 0ull);
            __syncwarp();
        }
        uint32_t *T32 = reinterpret_cast<uint32_t *>(T);
        if (x.type == T_ARRAY) {
            const uint16_t *v = reinterpret_cast<const uint16_t *>(x.p);
            for (uint32_t j = lane; j < x.card; j += 32) {
                const uint32_t y = __ldg(v + j);
                atomicOr(T32 + (y >> 5), 1u << (y & 31));
            }
        } else {
            const uint32_t *runs = reinterpret_cast<const uint32_t *>(x.p);
            for (uint32_t j = lane; j < x.runs; j += 32) {
                const uint32_t w = __ldg(runs + j), s = w & 0xFFFFu, e = s + (w >> 16);
                const uint32_t ws = s >> 5, we = e >> 5;
                const uint32_t ms = ~0u << (s & 31), me = ~0u >> (31 - (e & 31));
                if (ws == we) {
                    atomicOr(T32 + ws, ms & me);
                } else {
                    atomicOr(T32 + ws, ms);
                    for (uint32_t u = ws + 1; u < we; u++) T32[u] = ~0u;   // words inside one run
                    atomicOr(T32 + we, me);
                }
            }
        }
        __syncwarp();
    }
}

// AND with a later bitmap: every present key of the accumulator, 32 keys per
// warp step; the keys B lacks leave the map
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_acc_and(uint32_t *map, uint64_t *tiles, BmView B) {
    __shared__ __align__(16) uint64_t s_t[WARPS][1024];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *Ts = s_t[warp];
    const uint32_t warps = gridDim.x * WARPS;
    for (uint32_t k0 = (blockIdx.x * WARPS + warp) * 32; k0 < KEYS; k0 += warps * 32) {
        const uint32_t idx = map[k0 + lane];
        uint32_t m = __ballot_sync(FULL, idx != NO_TILE);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t key = k0 + src, ti = __shfl_sync(FULL, idx, src);
            const uint32_t j = lower_bound16(B.keys, B.n, key);
            const bool has = j < B.n && (uint32_t)__ldg(B.keys + j) == key;
            if (!has) {
                if (lane == 0) map[key] = NO_TILE;
                continue;
            }
            const CRef x = cref(B.base, __ldg(B.descs + j));
            const uint64_t *w = reinterpret_cast<const uint64_t *>(x.p);
            if (x.type != T_BITSET) {
                t_decode(Ts, x, lane);
                w = Ts;
            }
            ulonglong2 *T2 = reinterpret_cast<ulonglong2 *>(tiles + (size_t)ti * 1024);
            const ulonglong2 *W2 = reinterpret_cast<const ulonglong2 *>(w);
#pragma unroll 4
            for (int k = 0; k < 16; k++) {
                const ulonglong2 a = T2[32 * k + lane], b = W2[32 * k + lane];
                T2[32 * k + lane] = make_ulonglong2(a.x & b.x, a.y & b.y);
            }
            __syncwarp();
        }
    }
}

// per key: cardinality, runs and canonical type of its tile; words and
// bitset counts for the layout
__global__ void k_acc_count(const uint32_t *map, const uint64_t *tiles, uint64_t *info) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t k0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; k0 < KEYS; k0 += warps * 32) {
        const uint32_t idx = map[k0 + lane];
        info[k0 + lane] = ~0ull;
        __syncwarp();
        uint32_t m = __ballot_sync(FULL, idx != NO_TILE);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t ti = __shfl_sync(FULL, idx, src);
            const uint64_t *T = tiles + (size_t)ti * 1024;
            uint32_t c, r;
            t_combine<false>(nullptr, T, T, OP_OR, c, r, lane);
            if (lane == 0 && c) info[k0 + src] = pack_info(c, canon_type(c, r), canon_type(c, r) == T_RUN ? r : 0);
        }
    }
}

// exclusive scans over the 65536 keys: output index, word-region offset and
// bitset index of each present key; totals into st
__global__ void __launch_bounds__(1024) k_acc_scan(const uint64_t *info, uint32_t *pidx, uint64_t *woff,
                                                   uint32_t *bidx, AccState *st) {
    __shared__ unsigned long long s_w[32], s_c[32];
    __shared__ uint32_t s_p[32], s_b[32];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // thread t owns keys 64t .. 64t + 63
    uint32_t np = 0, nb = 0;
    unsigned long long nw = 0, card = 0;
    for (uint32_t k = 64 * t; k < 64 * t + 64; k++) {
        const uint64_t d = info[k];
        if (d == ~0ull) continue;
        const uint32_t c = (uint32_t)(d & 0xFFFFu) + 1, ty = (uint32_t)(d >> 16) & 3u, r = (uint32_t)(d >> 18) & 0x7FFu;
        np++;
        card += c;
        if (ty == T_BITSET) nb++;
        else nw += word_alloc_bytes(ty, c, r);
    }
    // block-wide exclusive scans of np, nb, nw
    uint32_t ip = warp_incl(np, lane), ib = warp_incl(nb, lane);
    unsigned long long iw = nw;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, iw, d);
        if (lane >= (uint32_t)d) iw += y;
    }
    const unsigned long long csum = warp_sum64(card);
    if (lane == 31) {
        s_p[warp] = ip;
        s_b[warp] = ib;
        s_w[warp] = iw;
    }
    if (lane == 0) s_c[warp] = csum;
    __syncthreads();
    if (warp == 0) {
        const uint32_t vp = s_p[lane], vb = s_b[lane];
        const unsigned long long vw = s_w[lane], vc = s_c[lane];
        const uint32_t xp = warp_incl(vp, lane), xb = warp_incl(vb, lane);
        unsigned long long xw = vw;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, xw, d);
            if (lane >= (uint32_t)d) xw += y;
        }
        const unsigned long long tc = warp_sum64(vc);
        s_p[lane] = xp - vp;
        s_b[lane] = xb - vb;
        s_w[lane] = xw - vw;
        if (lane == 31) {
            st->n_keys = xp;
            st->n_bits = xb;
            st->words = xw;
            st->card = tc;
        }
    }
    __syncthreads();
    uint32_t p = s_p[warp] + ip - np, b = s_b[warp] + ib - nb;
    unsigned long long w = s_w[warp] + iw - nw;
    for (uint32_t k = 64 * t; k < 64 * t + 64; k++) {
        const uint64_t d = info[k];
        if (d == ~0ull) continue;
        const uint32_t c = (uint32_t)(d & 0xFFFFu) + 1, ty = (uint32_t)(d >> 16) & 3u, r = (uint32_t)(d >> 18) & 0x7FFu;
        pidx[k] = p++;
        woff[k] = w;
        bidx[k] = b;
        if (ty == T_BITSET) b++;
        else w += word_alloc_bytes(ty, c, r);
    }
}

// write the canonical result: keys, descriptors and payloads
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_acc_emit(const uint32_t *map, const uint64_t *tiles, const uint64_t *info,
                                                         const uint32_t *pidx, const uint64_t *woff,
                                                         const uint32_t *bidx, uint8_t *base, uint16_t *okeys,
                                                         uint64_t *odescs, uint64_t words_off, uint64_t bits_off) {
    __shared__ __align__(16) uint16_t s_se[WARPS][4096];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t warps = gridDim.x * WARPS;
    for (uint32_t k0 = (blockIdx.x * WARPS + warp) * 32; k0 < KEYS; k0 += warps * 32) {
        const uint64_t d = info[k0 + lane];
        uint32_t m = __ballot_sync(FULL, d != ~0ull);
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t key = k0 + src;
            const uint64_t ds = __shfl_sync(FULL, d, src);
            const uint32_t c = (uint32_t)(ds & 0xFFFFu) + 1, ty = (uint32_t)(ds >> 16) & 3u, r = (uint32_t)(ds >> 18) & 0x7FFu;
            const uint64_t *T = tiles + (size_t)map[key] * 1024;
            uint64_t off;
            if (ty == T_BITSET) {
                off = bits_off + 8192ull * bidx[key];
                t_emit_bitset(T, reinterpret_cast<uint64_t *>(base + off), lane);
            } else {
                off = words_off + woff[key];
                if (ty == T_ARRAY) t_emit_array(T, reinterpret_cast<uint16_t *>(base + off), lane);
                else t_emit_runs(T, s_se[warp], s_se[warp] + 2048, reinterpret_cast<uint32_t *>(base + off), r, lane);
            }
            if (lane == 0) {
                okeys[pidx[key]] = (uint16_t)key;
                odescs[pidx[key]] = mk_desc(c, ty, r, off);
            }
            __syncwarp();
        }
    }
}

}  // namespace

struct rb_accum {
    uint32_t op, max_tiles;
    bool filled;          // AND: the first add has been applied
    uint8_t *dev;
    uint64_t bytes;
    uint32_t *map;
    AccState *st;
    uint64_t *info, *woff;
    uint32_t *pidx, *bidx;
    uint64_t *tiles;
};

namespace {

rb_status acc_clear(rb_accum *a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a->map, 0xFF, 4ull * KEYS, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->st, 0, sizeof(AccState), s);
    if (e != cudaSuccess) return cuda_err(e, "accumulator reset");
    a->filled = false;
    return RB_OK;
}

}  // namespace

extern "C" {

rb_status rb_accum_create(rb_op op, uint32_t max_keys, void *stream, rb_accum_t **out) {
    clear_stale_error();
    if (!out) return set_err(RB_EINVAL, "rb_accum_create: out is NULL");
    *out = nullptr;
    if (op != RB_AND && op != RB_OR) return set_err(RB_EINVAL, "rb_accum_create: op must be RB_AND or RB_OR");
    if (max_keys == 0 || max_keys > KEYS) return set_err(RB_EINVAL, "rb_accum_create: max_keys must be 1..65536");
    cudaStream_t s = (cudaStream_t)stream;
    rb_accum *a = new rb_accum;
    memset(a, 0, sizeof *a);
    a->op = op;
    a->max_tiles = max_keys;
    const uint64_t o_map = 0, o_st = align_up(4ull * KEYS, 256), o_info = align_up(o_st + sizeof(AccState), 256);
    const uint64_t o_woff = o_info + 8ull * KEYS, o_pidx = o_woff + 8ull * KEYS, o_bidx = o_pidx + 4ull * KEYS;
    const uint64_t o_tiles = align_up(o_bidx + 4ull * KEYS, 256);
    a->bytes = o_tiles + 8192ull * max_keys;
    a->dev = (uint8_t *)dev_alloc(a->bytes, s);
    if (!a->dev) { delete a; return RB_ENOMEM; }
    a->map = (uint32_t *)(a->dev + o_map);
    a->st = (AccState *)(a->dev + o_st);
    a->info = (uint64_t *)(a->dev + o_info);
    a->woff = (uint64_t *)(a->dev + o_woff);
    a->pidx = (uint32_t *)(a->dev + o_pidx);
    a->bidx = (uint32_t *)(a->dev + o_bidx);
    a->tiles = (uint64_t *)(a->dev + o_tiles);
    rb_status st = acc_clear(a, s);
    if (st != RB_OK) { dev_free(a->dev, a->bytes, s); delete a; return st; }
    *out = a;
    return RB_OK;
}

rb_status rb_accum_add(rb_accum_t *a, const rb_t *b, void *stream) {
    clear_stale_error();
    if (!a || !b) return set_err(RB_EINVAL, "rb_accum_add: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const BmView B = view_of(b);
    const unsigned cap = (unsigned)sm_count() * 8;
    if (a->op == RB_OR || !a->filled) {
        if (B.n) {
            const unsigned need = (B.n + 7) / 8;
            k_acc_or<<<need < cap ? need : cap, 256, 0, s>>>(a->map, a->tiles, a->st, a->max_tiles, B);
        }
        a->filled = true;
    } else {
        k_acc_and<4><<<std::min<unsigned>(KEYS / 128, (unsigned)sm_count() * 4), 128, 0, s>>>(a->map, a->tiles, B);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "rb_accum_add");
    return RB_OK;
}

rb_status rb_accum_result(rb_accum_t *a, rb_t **out, uint64_t *card, void *stream) {
    clear_stale_error();
    if (out) *out = nullptr;
    if (!a) return set_err(RB_EINVAL, "rb_accum_result: NULL accumulator");
    cudaStream_t s = (cudaStream_t)stream;
    AccState *h = (AccState *)pinned_scratch(sizeof(AccState));
    if (!h) return set_err(RB_ENOMEM, "pinned staging allocation failed");
    k_acc_count<<<(unsigned)sm_count() * 4, 256, 0, s>>>(a->map, a->tiles, a->info);
    k_acc_scan<<<1, 1024, 0, s>>>(a->info, a->pidx, a->woff, a->bidx, a->st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, a->st, sizeof(AccState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e, "rb_accum_result");
    if (h->status & 1u)
        return set_err(RB_ERANGE, "rb_accum: more keys than the %u tiles reserved at creation", a->max_tiles);
    if (card) *card = h->card;
    if (!out) return RB_OK;
    const uint32_t n = h->n_keys;
    const uint64_t descs_off = align_up(2ull * n, 256), words_off = align_up(descs_off + 8ull * n, 256);
    const uint64_t bits_off = align_up(words_off + h->words, 256), total = std::max<uint64_t>(bits_off + 8192ull * h->n_bits, 16);
    rb *r = handle_new();
    r->arena = arena_new(total, s);
    if (!r->arena) { delete r; return RB_ENOMEM; }
    r->base = (uint8_t *)r->arena->ptr;
    r->keys = (uint16_t *)r->base;
    r->descs = (uint64_t *)(r->base + descs_off);
    r->n = n;
    r->card = h->card;
    r->word_bytes = h->words;
    r->n_bitsets = h->n_bits;
    if (n) {
        k_acc_emit<4><<<std::min<unsigned>(KEYS / 128, (unsigned)sm_count() * 4), 128, 0, s>>>(
            a->map, a->tiles, a->info, a->pidx, a->woff, a->bidx, r->base, r->keys, r->descs, words_off, bits_off);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rb_free(r);
            return cuda_err(e, "rb_accum_result emit");
        }
    }
    *out = r;
    return RB_OK;
}

rb_status rb_accum_reset(rb_accum_t *a, void *stream) {
    if (!a) return set_err(RB_EINVAL, "rb_accum_reset: NULL accumulator");
    return acc_clear(a, (cudaStream_t)stream);
}

void rb_accum_free(rb_accum_t *a) {
    if (!a) return;
    cudaDeviceSynchronize();   // adds may still be running on any stream
    dev_free(a->dev, a->bytes, nullptr);
    delete a;
}

}  // extern "C"
