// rb_core.cu - handles, memory, errors, construction, decode and layout export.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "rb_device.cuh"

using namespace rbi;
using namespace rbd;

// ------------------------------------------------------------------ errors

namespace {
thread_local char g_err[512] = "";
std::mutex g_alloc_mu;
rb_alloc_fn g_alloc = nullptr;
rb_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
rb_schedule g_sched = {4, 3, 96, 0, 0, 32};
std::mutex g_sched_mu;
}  // namespace

namespace rbi {

rb_status set_err(rb_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

rb_status cuda_err(cudaError_t e, const char *what) {
    return set_err(RB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dev_alloc(uint64_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    rb_alloc_fn fa;
    void *ctx;
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        fa = g_alloc;
        ctx = g_alloc_ctx;
    }
    void *p = nullptr;
    if (fa) {
        p = fa(bytes, (void *)s, ctx);
    } else if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (!p) set_err(RB_ENOMEM, "device allocation of %llu bytes failed", (unsigned long long)bytes);
    return p;
}

void dev_free(void *p, uint64_t bytes, cudaStream_t s) {
    if (!p) return;
    rb_free_fn ff;
    void *ctx;
    {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        ff = g_free;
        ctx = g_alloc_ctx;
    }
    if (ff) ff(p, bytes ? bytes : 16, (void *)s, ctx);
    else cudaFreeAsync(p, s);
}

void *dev_alloc_native(uint64_t bytes, cudaStream_t s) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes ? bytes : 16, s) != cudaSuccess) {
        cudaGetLastError();
        set_err(RB_ENOMEM, "device allocation of %llu bytes failed", (unsigned long long)bytes);
        return nullptr;
    }
    return p;
}
void dev_free_native(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

static RbArena *arena_wrap(void *p, uint64_t bytes, cudaStream_t s, int native) {
    RbArena *a = new RbArena;
    a->ptr = p;
    a->bytes = bytes ? bytes : 16;
    a->stream = s;
    a->refs.store(1);
    a->native = native;
    a->budget = nullptr;
    a->charge = 0;
    return a;
}
RbArena *arena_new(uint64_t bytes, cudaStream_t s) {
    void *p = dev_alloc(bytes, s);
    return p ? arena_wrap(p, bytes, s, 0) : nullptr;
}
RbArena *arena_new_native(uint64_t bytes, cudaStream_t s) {
    void *p = dev_alloc_native(bytes, s);
    return p ? arena_wrap(p, bytes, s, 1) : nullptr;
}
void arena_ref(RbArena *a) {
    if (a) a->refs.fetch_add(1);
}
void budget_unref(RbBudget *b) {
    if (b && b->refs.fetch_sub(1) == 1) delete b;
}
void arena_unref(RbArena *a) { arena_unref_n(a, 1); }
void arena_unref_n(RbArena *a, int n) {
    if (a && n > 0 && a->refs.fetch_sub(n) == n) {
        if (a->native) dev_free_native(a->ptr, a->stream);
        else dev_free(a->ptr, a->bytes, a->stream);
        if (a->budget) {
            a->budget->used.fetch_sub((int64_t)a->charge);
            {
                std::lock_guard<std::mutex> g(a->budget->mu);
                if (a->budget->notify) a->budget->notify(a->budget->ctx);
            }
            budget_unref(a->budget);
        }
        delete a;
    }
}

void *pinned_scratch(uint64_t bytes) {
    struct Buf {
        void *p = nullptr;
        uint64_t n = 0;
        ~Buf() {
            if (p) cudaFreeHost(p);
        }
    };
    static thread_local Buf buf;
    if (bytes > buf.n) {
        if (buf.p) cudaFreeHost(buf.p);
        uint64_t n = align_up(bytes, 1 << 20);
        if (cudaMallocHost(&buf.p, n) != cudaSuccess) {
            cudaGetLastError();
            buf.p = nullptr;
            buf.n = 0;
            return nullptr;
        }
        buf.n = n;
    }
    return buf.p;
}

// SM count of the current device, looked up once per device; concurrent
// first calls store the same value
int sm_count() {
    constexpr int MAX_DEV = 256;
    static std::atomic<int> cache[MAX_DEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    int n = dev < MAX_DEV ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    if (dev < MAX_DEV) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

BmView view_of(const rb *b) {
    BmView v;
    v.keys = b->keys;
    v.descs = b->descs;
    v.base = b->base;
    v.n = b->n;
    v.pad = 0;
    return v;
}

rb *handle_new() {
    rb *h = new rb;
    memset(h, 0, sizeof *h);
    return h;
}

rb_schedule current_schedule() {
    std::lock_guard<std::mutex> g(g_sched_mu);
    return g_sched;
}

}  // namespace rbi

// ------------------------------------------------------------ construction

namespace {

struct BuildTotals {
    unsigned int err;        // 1: input not strictly increasing
    unsigned int n;          // containers
    unsigned long long words;
    unsigned int bitsets;
    unsigned int pad;
};

// per value: chunk key and whether it starts a run; warp-aggregated counts of
// values and run starts per key (values are sorted, so equal keys are
// contiguous within a warp)
__global__ void k_build_count(const uint32_t *__restrict__ v, uint64_t n, uint32_t *cnt, uint32_t *runs,
                              BuildTotals *tot) {
    const uint32_t lane = threadIdx.x & 31;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        uint64_t i = base + lane;
        uint32_t key = 0x10000u, rs = 0;
        if (i < n) {
            uint32_t x = __ldg(v + i);
            key = x >> 16;
            if (i == 0) {
                rs = 1;
            } else {
                uint32_t p = __ldg(v + i - 1);
                if (x <= p) atomicOr(&tot->err, 1u);
                rs = (x != p + 1) || ((p >> 16) != key);
            }
        }
        uint32_t grp = __match_any_sync(FULL, key);
        uint32_t starts = __ballot_sync(FULL, rs);
        if (i < n && lane == (uint32_t)(__ffs(grp) - 1)) {
            atomicAdd(cnt + key, (uint32_t)__popc(grp));
            atomicAdd(runs + key, (uint32_t)__popc(grp & starts));
        }
    }
}

// one block of 1024 threads over the 65536 possible keys (64 consecutive keys
// per thread): canonical type per key, then scans for the container index,
// word-region offset, bitset index and first value of each container
__global__ void __launch_bounds__(1024) k_build_plan(const uint32_t *cnt, const uint32_t *runs, uint16_t *tkeys,
                                                     uint64_t *tinfo, uint64_t *tvstart, BuildTotals *tot) {
    __shared__ uint32_t s_n[32], s_b[32];
    __shared__ unsigned long long s_w[32], s_v[32];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t ln = 0, lb = 0;
    unsigned long long lw = 0, lv = 0;
    for (uint32_t k = t * 64; k < t * 64 + 64; k++) {
        uint32_t c = cnt[k];
        if (!c) continue;
        uint32_t ty = canon_type(c, runs[k]);
        ln++;
        lv += c;
        if (ty == T_BITSET) lb++;
        else lw += word_alloc_bytes(ty, c, runs[k]);
    }
    // block exclusive scans of (ln, lb, lw, lv)
    uint32_t in = warp_incl(ln, lane), ib = warp_incl(lb, lane);
    unsigned long long iw = lw, iv = lv;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long yw = __shfl_up_sync(FULL, iw, d), yv = __shfl_up_sync(FULL, iv, d);
        if (lane >= (uint32_t)d) { iw += yw; iv += yv; }
    }
    if (lane == 31) { s_n[warp] = in; s_b[warp] = ib; s_w[warp] = iw; s_v[warp] = iv; }
    __syncthreads();
    if (warp == 0) {
        uint32_t a = s_n[lane], b = s_b[lane];
        unsigned long long w = s_w[lane], vv = s_v[lane];
        uint32_t ia = warp_incl(a, lane), ibb = warp_incl(b, lane);
        unsigned long long iww = w, ivv = vv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned long long yw = __shfl_up_sync(FULL, iww, d), yv = __shfl_up_sync(FULL, ivv, d);
            if (lane >= (uint32_t)d) { iww += yw; ivv += yv; }
        }
        s_n[lane] = ia - a; s_b[lane] = ibb - b; s_w[lane] = iww - w; s_v[lane] = ivv - vv;
        if (lane == 31) {
            tot->n = ia;
            tot->bitsets = ibb;
            tot->words = iww;
        }
    }
    __syncthreads();
    uint32_t on = s_n[warp] + in - ln, ob = s_b[warp] + ib - lb;
    unsigned long long ow = s_w[warp] + iw - lw, ov = s_v[warp] + iv - lv;
    for (uint32_t k = t * 64; k < t * 64 + 64; k++) {
        uint32_t c = cnt[k];
        if (!c) continue;
        uint32_t r = runs[k], ty = canon_type(c, r);
        tkeys[on] = (uint16_t)k;
        // info: card, type, runs, and the offset within the word region or
        // the bitset index (resolved to bytes once the region sizes are known)
        uint64_t where = ty == T_BITSET ? ob : ow;
        tinfo[on] = (uint64_t)(c - 1) | ((uint64_t)ty << 16) | ((uint64_t)(ty == T_RUN ? r : 0) << 18) |
                    (where << 29);
        tvstart[on] = ov;
        on++;
        ov += c;
        if (ty == T_BITSET) ob++;
        else ow += word_alloc_bytes(ty, c, r);
    }
}

// one warp per container: write its payload and final descriptor
__global__ void k_build_fill(const uint32_t *__restrict__ v, const uint16_t *tkeys, const uint64_t *tinfo,
                             const uint64_t *tvstart, uint32_t n, uint16_t *keys, uint64_t *descs, uint8_t *base,
                             uint64_t words_off, uint64_t bits_off) {
    extern __shared__ __align__(16) uint64_t smem[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    uint64_t *T = smem + warp * 1024;
    for (uint32_t ci = blockIdx.x * wpb + warp; ci < n; ci += gridDim.x * wpb) {
        uint64_t info = tinfo[ci];
        uint32_t c = (uint32_t)(info & 0xFFFF) + 1, ty = (uint32_t)(info >> 16) & 3, r = (uint32_t)(info >> 18) & 0x7FF;
        uint64_t where = info >> 29;
        uint64_t off = ty == T_BITSET ? bits_off + where * 8192ull : words_off + where;
        const uint32_t *src = v + tvstart[ci];
        uint8_t *dst = base + off;
        if (ty == T_ARRAY) {
            uint16_t *o = reinterpret_cast<uint16_t *>(dst);
            for (uint32_t i = lane; i < c; i += 32) o[i] = (uint16_t)(__ldg(src + i) & 0xFFFFu);
        } else if (ty == T_BITSET) {
            t_zero(T, lane);
            __syncwarp();
            uint32_t *T32 = reinterpret_cast<uint32_t *>(T);
            for (uint32_t i = lane; i < c; i += 32) {
                uint32_t x = __ldg(src + i) & 0xFFFFu;
                atomicOr(T32 + (x >> 5), 1u << (x & 31));
            }
            __syncwarp();
            t_emit_bitset(T, reinterpret_cast<uint64_t *>(dst), lane);
            __syncwarp();
        } else {
            // run starts in value order; run k = [v[s_k], v[s_{k+1} - 1]]
            uint32_t *o = reinterpret_cast<uint32_t *>(dst);
            uint32_t b = 0;
            for (uint32_t i0 = 0; i0 < c; i0 += 32) {
                uint32_t i = i0 + lane;
                uint32_t st = 0;
                if (i < c) st = (i == 0) || (__ldg(src + i) != __ldg(src + i - 1) + 1);
                uint32_t m = __ballot_sync(FULL, st);
                if (st) o[b + __popc(m & lanemask_lt(lane))] = i;
                b += __popc(m);
            }
            __syncwarp();
            for (uint32_t k0 = 0; k0 < r; k0 += 32) {
                uint32_t k = k0 + lane, s = 0, e = 0;
                if (k < r) {
                    s = o[k];
                    e = (k + 1 < r ? o[k + 1] : c) - 1;
                }
                __syncwarp();
                if (k < r) {
                    uint32_t lo = __ldg(src + s) & 0xFFFFu, hi = __ldg(src + e) & 0xFFFFu;
                    o[k] = lo | ((hi - lo) << 16);
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            keys[ci] = tkeys[ci];
            descs[ci] = mk_desc(c, ty, ty == T_RUN ? r : 0, off);
        }
    }
}

// exclusive prefix of container cardinalities (n <= 65536), 1024 threads
__global__ void __launch_bounds__(1024) k_scan_cards(const uint64_t *descs, uint32_t n, uint64_t *offs) {
    __shared__ unsigned long long s[32];
    const uint32_t t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t per = (n + 1023) / 1024;
    unsigned long long loc = 0;
    for (uint32_t i = t * per; i < min(n, t * per + per); i++) loc += d_card(descs[i]);
    unsigned long long inc = loc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        unsigned long long y = __shfl_up_sync(FULL, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    if (lane == 31) s[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = s[lane], xi = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            unsigned long long y = __shfl_up_sync(FULL, xi, d);
            if (lane >= (uint32_t)d) xi += y;
        }
        s[lane] = xi - x;
    }
    __syncthreads();
    unsigned long long o = s[warp] + inc - loc;
    for (uint32_t i = t * per; i < min(n, t * per + per); i++) {
        offs[i] = o;
        o += d_card(descs[i]);
    }
}

// one warp per container: expand to key << 16 | low values
__global__ void k_decode(const uint16_t *keys, const uint64_t *descs, const uint8_t *base, uint32_t n,
                         const uint64_t *offs, uint32_t *out) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (uint32_t ci = blockIdx.x * wpb + warp; ci < n; ci += gridDim.x * wpb) {
        uint64_t d = descs[ci];
        CRef x = cref(base, d);
        uint32_t hi = (uint32_t)keys[ci] << 16;
        uint32_t *o = out + offs[ci];
        if (x.type == T_ARRAY) {
            const uint16_t *a = reinterpret_cast<const uint16_t *>(x.p);
            for (uint32_t i = lane; i < x.card; i += 32) o[i] = hi | a[i];
        } else if (x.type == T_RUN) {
            const uint32_t *rr = reinterpret_cast<const uint32_t *>(x.p);
            uint32_t pos = 0;
            for (uint32_t k = 0; k < x.runs; k++) {
                uint32_t w = rr[k], s = w & 0xFFFFu, len = (w >> 16) + 1;
                for (uint32_t i = lane; i < len; i += 32) o[pos + i] = hi | (s + i);
                pos += len;
            }
        } else {
            const ulonglong2 *W = reinterpret_cast<const ulonglong2 *>(x.p);
            uint32_t b = 0;
            for (int k = 0; k < 16; k++) {
                ulonglong2 w = W[32 * k + lane];
                uint32_t cnt = __popcll(w.x) + __popcll(w.y);
                uint32_t inc = warp_incl(cnt, lane);
                uint32_t pos = b + inc - cnt;
                b += __shfl_sync(FULL, inc, 31);
                uint32_t v0 = (uint32_t)(64 * k + 2 * lane) * 64u;
                uint64_t y = w.x;
                while (y) { o[pos++] = hi | (v0 + __ffsll((long long)y) - 1); y &= y - 1; }
                y = w.y;
                while (y) { o[pos++] = hi | (v0 + 64 + __ffsll((long long)y) - 1); y &= y - 1; }
            }
        }
    }
}

// one warp per container: copy its payload bytes to the packed export buffer
__global__ void k_gather(const uint64_t *descs, const uint8_t *base, uint32_t n, const uint64_t *offs,
                         uint8_t *out) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    for (uint32_t ci = blockIdx.x * wpb + warp; ci < n; ci += gridDim.x * wpb) {
        uint64_t d = descs[ci];
        const uint8_t *src = base + d_off(d);
        uint8_t *dst = out + offs[ci];
        uint32_t bytes = (uint32_t)(offs[ci + 1] - offs[ci]);
        const uint16_t *s16 = reinterpret_cast<const uint16_t *>(src);
        uint16_t *d16 = reinterpret_cast<uint16_t *>(dst);
        for (uint32_t i = lane; i < bytes / 2; i += 32) d16[i] = s16[i];
    }
}

}  // namespace

namespace rbi {

// Enqueue the decode of b (b->n > 0) into device memory `out` on stream s,
// with the per-container output offsets in caller-provided device memory
// `offs` (at least b->n entries).  No allocation, no synchronisation.
cudaError_t enqueue_decode(const rb *b, uint64_t *offs, uint32_t *out, cudaStream_t s) {
    k_scan_cards<<<1, 1024, 0, s>>>(b->descs, b->n, offs);
    const uint32_t grid = (b->n + 7) / 8, gcap = (uint32_t)sm_count() * 8;
    k_decode<<<grid < gcap ? grid : gcap, 256, 0, s>>>(b->keys, b->descs, b->base, b->n, offs, out);
    return cudaGetLastError();
}

}  // namespace rbi

extern "C" {

const char *rb_last_error(void) { return g_err; }

const char *rb_version(void) { return "gbroaring 0.1 (sm_103a)"; }

rb_status rb_set_allocator(rb_alloc_fn alloc, rb_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return set_err(RB_EINVAL, "rb_set_allocator: give both hooks or neither");
    std::lock_guard<std::mutex> g(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return RB_OK;
}

rb_status rb_set_schedule(const rb_schedule *s) {
    if (!s) return set_err(RB_EINVAL, "rb_set_schedule: NULL");
    if (!(s->warps_per_cta == 2 || s->warps_per_cta == 4 || s->warps_per_cta == 8))
        return set_err(RB_EINVAL, "warps_per_cta must be 2, 4 or 8");
    if (s->ctas_per_sm < 1 || s->ctas_per_sm * s->warps_per_cta * 16384u > 228u * 1024u)
        return set_err(RB_EINVAL, "ctas_per_sm out of range for 16 KB of tiles per warp");
    if (s->small_intervals > 2047) return set_err(RB_EINVAL, "small_intervals must be <= 2047");
    if (s->lean_ctas_per_sm > 8) return set_err(RB_EINVAL, "lean_ctas_per_sm must be <= 8");
    if (s->prefetch_lines > 64) return set_err(RB_EINVAL, "prefetch_lines must be <= 64");
    if (s->tiles_per_take > 256) return set_err(RB_EINVAL, "tiles_per_take must be <= 256");
    std::lock_guard<std::mutex> g(g_sched_mu);
    g_sched = *s;
    return RB_OK;
}

rb_status rb_get_schedule(rb_schedule *s) {
    if (!s) return set_err(RB_EINVAL, "rb_get_schedule: NULL");
    *s = current_schedule();
    return RB_OK;
}

static void block_unref(RbBlock *k, uint64_t n) {
    if (k->refs.fetch_sub(n) == n) {
        delete[] k->items;
        delete k;
    }
}

void rb_free(rb_t *b) {
    if (!b) return;
    arena_unref(b->arena);
    if (b->block) block_unref(b->block, 1);
    else delete b;
}

void rb_free_array(rb_t *const *hs, uint64_t n) {
    if (!hs) return;
    // runs of handles that share an arena and a block (the results of one
    // batch) give back their references in one step each
    uint64_t i = 0;
    while (i < n) {
        rb *h = hs[i];
        if (!h) { i++; continue; }
        if (!h->block) { rb_free(h); i++; continue; }
        RbArena *a = h->arena;
        RbBlock *k = h->block;
        uint64_t j = i + 1;
        while (j < n && hs[j] && hs[j]->block == k && hs[j]->arena == a) j++;
        // the run holds j - i references of each; the block is released last
        uint64_t left = j - i;
        while (left) {
            const int step = (int)std::min<uint64_t>(left, 1u << 30);
            arena_unref_n(a, step);
            left -= (uint64_t)step;
        }
        block_unref(k, j - i);
        i = j;
    }
}

rb_status rb_cardinality(const rb_t *b, uint64_t *out) {
    if (!b || !out) return set_err(RB_EINVAL, "rb_cardinality: NULL argument");
    *out = b->card;
    return RB_OK;
}

rb_status rb_from_sorted_u32(const uint32_t *vals, uint64_t n, int vals_on_device, void *stream, rb_t **out) {
    clear_stale_error();
    if (!out) return set_err(RB_EINVAL, "rb_from_sorted_u32: out is NULL");
    *out = nullptr;
    if (n && !vals) return set_err(RB_EINVAL, "rb_from_sorted_u32: vals is NULL");
    if (n > (1ull << 32)) return set_err(RB_ERANGE, "rb_from_sorted_u32: more than 2^32 values");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        rb *h = handle_new();
        h->arena = arena_new(16, s);
        if (!h->arena) { delete h; return RB_ENOMEM; }
        h->base = (uint8_t *)h->arena->ptr;
        *out = h;
        return RB_OK;
    }
    // temporaries: [values if on host][cnt 256K][runs 256K][tkeys 128K][tinfo 512K][tvstart 512K][totals]
    const uint64_t vbytes = vals_on_device ? 0 : align_up(n * 4, 256);
    const uint64_t tmp_bytes = vbytes + 65536ull * (4 + 4 + 2 + 8 + 8) + 256;
    uint8_t *tmp = (uint8_t *)dev_alloc(tmp_bytes, s);
    if (!tmp) return RB_ENOMEM;
    rb_status st = RB_OK;
    const uint32_t *dv = vals;
    uint32_t *cnt = (uint32_t *)(tmp + vbytes);
    uint32_t *runs = cnt + 65536;
    uint16_t *tkeys = (uint16_t *)(runs + 65536);
    uint64_t *tinfo = (uint64_t *)(tkeys + 65536);
    uint64_t *tvstart = tinfo + 65536;
    BuildTotals *tot = (BuildTotals *)(tvstart + 65536);
    BuildTotals *htot = (BuildTotals *)pinned_scratch(sizeof(BuildTotals));
    rb *h = nullptr;
    do {
        if (!htot) { st = set_err(RB_ENOMEM, "pinned staging allocation failed"); break; }
        cudaError_t e;
        if (!vals_on_device) {
            e = cudaMemcpyAsync(tmp, vals, n * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { st = cuda_err(e, "copy values to device"); break; }
            dv = (const uint32_t *)tmp;
        }
        e = cudaMemsetAsync(cnt, 0, 65536ull * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(tot, 0, sizeof(BuildTotals), s);
        if (e != cudaSuccess) { st = cuda_err(e, "memset"); break; }
        uint64_t blocks = (n + 255) / 256;
        uint64_t cap = (uint64_t)sm_count() * 8;
        k_build_count<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(dv, n, cnt, runs, tot);
        k_build_plan<<<1, 1024, 0, s>>>(cnt, runs, tkeys, tinfo, tvstart, tot);
        e = cudaMemcpyAsync(htot, tot, sizeof(BuildTotals), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = cuda_err(e, "build count"); break; }
        if (htot->err) { st = set_err(RB_EINVAL, "rb_from_sorted_u32: input is not strictly increasing"); break; }
        const uint32_t nc = htot->n;
        const uint64_t words = htot->words;
        const uint32_t nbits = htot->bitsets;
        const uint64_t keys_off = 0, descs_off = align_up(2ull * nc, 256);
        const uint64_t words_off = align_up(descs_off + 8ull * nc, 256);
        const uint64_t bits_off = align_up(words_off + words, 256);
        const uint64_t total = bits_off + 8192ull * nbits;
        if (total >= MAX_OFFSET) { st = set_err(RB_ERANGE, "bitmap larger than the 128 GiB descriptor reach"); break; }
        h = handle_new();
        h->arena = arena_new(total, s);
        if (!h->arena) { delete h; h = nullptr; st = RB_ENOMEM; break; }
        h->base = (uint8_t *)h->arena->ptr;
        h->keys = (uint16_t *)(h->base + keys_off);
        h->descs = (uint64_t *)(h->base + descs_off);
        h->n = nc;
        h->card = n;
        h->word_bytes = words;
        h->n_bitsets = nbits;
        const int wpb = 4;
        uint32_t grid = (nc + wpb - 1) / wpb;
        uint32_t gcap = (uint32_t)sm_count() * 8;
        k_build_fill<<<grid < gcap ? grid : gcap, wpb * 32, wpb * 8192, s>>>(
            dv, tkeys, tinfo, tvstart, nc, h->keys, h->descs, h->base, words_off, bits_off);
        e = cudaGetLastError();
        if (e != cudaSuccess) { st = cuda_err(e, "build fill launch"); break; }
    } while (0);
    dev_free(tmp, tmp_bytes, s);
    if (st != RB_OK) {
        if (h) rb_free(h);
        return st;
    }
    *out = h;
    return RB_OK;
}

rb_status rb_info(const rb_t *b, uint32_t *n_containers, uint64_t *payload) {
    if (!b) return set_err(RB_EINVAL, "rb_info: NULL handle");
    if (n_containers) *n_containers = b->n;
    if (payload) {
        // export sizes: arrays 2c (allocation rounds to 4), runs 4r, bitsets 8192
        if (b->n == 0) { *payload = 0; return RB_OK; }
        std::vector<uint64_t> d(b->n);
        cudaError_t e = cudaMemcpy(d.data(), b->descs, 8ull * b->n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(e, "rb_info");
        uint64_t s = 0;
        for (uint64_t x : d) s += payload_bytes(d_type(x), d_card(x), d_runs(x));
        *payload = s;
    }
    return RB_OK;
}

rb_status rb_to_u32(const rb_t *b, uint32_t *dst, int dst_on_device, uint64_t cap, uint64_t *n_out, void *stream) {
    clear_stale_error();
    if (!b) return set_err(RB_EINVAL, "rb_to_u32: NULL handle");
    if (n_out) *n_out = b->card;
    if (b->card == 0) return RB_OK;
    if (!dst) return set_err(RB_EINVAL, "rb_to_u32: dst is NULL");
    if (cap < b->card) return set_err(RB_ERANGE, "rb_to_u32: capacity %llu below cardinality %llu",
                                      (unsigned long long)cap, (unsigned long long)b->card);
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t obytes = dst_on_device ? 0 : align_up(b->card * 4, 256);
    uint64_t tbytes = obytes + 8ull * b->n + 16;
    uint8_t *tmp = (uint8_t *)dev_alloc(tbytes, s);
    if (!tmp) return RB_ENOMEM;
    uint32_t *o = dst_on_device ? dst : (uint32_t *)tmp;
    uint64_t *offs = (uint64_t *)(tmp + obytes);
    k_scan_cards<<<1, 1024, 0, s>>>(b->descs, b->n, offs);
    uint32_t grid = (b->n + 7) / 8, gcap = (uint32_t)sm_count() * 8;
    k_decode<<<grid < gcap ? grid : gcap, 256, 0, s>>>(b->keys, b->descs, b->base, b->n, offs, o);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dst_on_device) e = cudaMemcpyAsync(dst, o, b->card * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(tmp, tbytes, s);
    if (e != cudaSuccess) return cuda_err(e, "rb_to_u32");
    return RB_OK;
}

rb_status rb_export_layout(const rb_t *b, uint16_t *keys, uint8_t *types, uint32_t *cards, uint64_t *offs,
                           uint8_t *payload, uint64_t payload_cap, void *stream) {
    clear_stale_error();
    if (!b) return set_err(RB_EINVAL, "rb_export_layout: NULL handle");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = b->n;
    std::vector<uint64_t> d(n);
    std::vector<uint16_t> k(n);
    if (n) {
        cudaError_t e = cudaMemcpyAsync(d.data(), b->descs, 8ull * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(k.data(), b->keys, 2ull * n, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(e, "rb_export_layout");
    }
    std::vector<uint64_t> o(n + 1);
    o[0] = 0;
    for (uint32_t i = 0; i < n; i++) o[i + 1] = o[i] + payload_bytes(d_type(d[i]), d_card(d[i]), d_runs(d[i]));
    if (offs) memcpy(offs, o.data(), 8ull * (n + 1));
    for (uint32_t i = 0; i < n; i++) {
        if (keys) keys[i] = k[i];
        if (types) types[i] = (uint8_t)d_type(d[i]);
        if (cards) cards[i] = d_card(d[i]);
    }
    if (!payload || n == 0) return RB_OK;
    if (payload_cap < o[n]) return set_err(RB_ERANGE, "rb_export_layout: payload capacity too small");
    uint64_t tb = align_up(8ull * (n + 1), 256) + o[n] + 16;
    uint8_t *tmp = (uint8_t *)dev_alloc(tb, s);
    if (!tmp) return RB_ENOMEM;
    uint64_t *doffs = (uint64_t *)tmp;
    uint8_t *dpay = tmp + align_up(8ull * (n + 1), 256);
    cudaError_t e = cudaMemcpyAsync(doffs, o.data(), 8ull * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        uint32_t grid = (n + 7) / 8, gcap = (uint32_t)sm_count() * 8;
        k_gather<<<grid < gcap ? grid : gcap, 256, 0, s>>>(b->descs, b->base, n, doffs, dpay);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(payload, dpay, o[n], cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(tmp, tb, s);
    if (e != cudaSuccess) return cuda_err(e, "rb_export_layout");
    return RB_OK;
}

}  // extern "C"
