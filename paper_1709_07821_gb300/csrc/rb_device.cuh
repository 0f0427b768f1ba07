// rb_device.cuh - warp-level building blocks shared by the container kernels.
//
// A "tile" is one container expanded to its 2^16-bit bitset in shared memory
// (1024 u64 words, 8 KB).  Lane l of a warp owns words 64k + 2l and 64k + 2l + 1
// for k = 0..15, read and written as 16-byte vectors, so every tile pass is a
// conflict-free sweep.  Each container kernel warp owns two tiles (T0, T1).
#pragma once

#include "rb_internal.h"

namespace rbd {
using namespace rbi;

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint64_t ALLOC_FAIL = ~0ull;
enum : uint32_t { OP_AND = 0, OP_OR = 1, OP_ANDNOT = 2, OP_XOR = 3 };

__device__ __forceinline__ uint32_t lanemask_lt(uint32_t lane) { return (1u << lane) - 1u; }

// ------------------------------------------------------------ bulk copies
// One lane moves a whole 8 KB bitset between global and shared memory with
// the bulk-copy (TMA) engine: loads complete on a per-warp mbarrier that the
// warp waits on (with an iteration limit), stores are tracked as bulk groups.
// Addresses are 16-byte aligned and sizes multiples of 16 (bitsets are 8 KB
// at 16-byte aligned offsets).

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's generic-proxy shared-memory accesses with the bulk-copy engine's
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst_smem)),
                 "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// wait until every bulk store of this thread has read its shared-memory source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until every bulk store of this thread has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity to complete: gives up
// after about one second of SM clock (2^31 cycles) and returns false (the
// caller records the error and stops using the tiles)
constexpr long long MBAR_WAIT_CYCLES = 1ll << 31;
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    return mbar_wait_for(bar, parity, MBAR_WAIT_CYCLES);
}

// 4 bytes from global to shared memory without holding a register
// (cp.async, Ampere onward); every copy a thread issued is complete once it
// has run cp_async_wait_all, which waits like a load does (no spin)
__device__ __forceinline__ void cp_async4(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
    return x;
}
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(FULL, x, d);
    return x;
}
__device__ __forceinline__ uint32_t warp_incl(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    return x;
}
__device__ __forceinline__ uint32_t warp_xor_incl(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, d);
        if (lane >= (uint32_t)d) x ^= y;
    }
    return x;
}

// first index i in sorted keys[0..n) with keys[i] >= key
__device__ __forceinline__ uint32_t lower_bound16(const uint16_t *keys, uint32_t n, uint32_t key) {
    uint32_t lo = 0, hi = n;
#pragma unroll 1
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if ((uint32_t)__ldg(keys + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------ containers

struct CRef {
    const uint8_t *p;
    uint32_t type, card, runs;
};
__device__ __forceinline__ CRef cref(const uint8_t *base, uint64_t d) {
    CRef c;
    c.p = base + d_off(d);
    c.type = d_type(d);
    c.card = d_card(d);
    c.runs = d_runs(d);
    return c;
}
// number of intervals a container contributes to a sweep (values of an
// array, runs of a run container); bitsets are never swept
__device__ __forceinline__ uint32_t n_intervals(uint64_t d) {
    uint32_t t = d_type(d);
    return t == T_ARRAY ? d_card(d) : t == T_RUN ? d_runs(d) : 0x100000u;
}
__device__ __forceinline__ uint32_t in_payload_bytes(uint64_t d) {
    return payload_bytes(d_type(d), d_card(d), d_runs(d));
}

__device__ __forceinline__ uint64_t apply_op(uint32_t op, uint64_t a, uint64_t b) {
    switch (op) {
        case OP_AND: return a & b;
        case OP_OR: return a | b;
        case OP_ANDNOT: return a & ~b;
        default: return a ^ b;
    }
}
// the op as a truth table over (in a, in b): masks m11, m10, m01 are all ones
// when the result holds a value present in both, only in a, only in b
struct OpMasks {
    uint64_t m11, m10, m01;
};
__device__ __forceinline__ OpMasks op_masks(uint32_t op) {
    OpMasks m;
    m.m11 = (op == OP_AND || op == OP_OR) ? ~0ull : 0ull;
    m.m10 = (op != OP_AND) ? ~0ull : 0ull;
    m.m01 = (op == OP_OR || op == OP_XOR) ? ~0ull : 0ull;
    return m;
}
__device__ __forceinline__ uint64_t apply_masks(const OpMasks &m, uint64_t a, uint64_t b) {
    return (a & b & m.m11) | (a & ~b & m.m10) | (~a & b & m.m01);
}
__device__ __forceinline__ bool member(uint32_t op, bool ina, bool inb) {
    switch (op) {
        case OP_AND: return ina && inb;
        case OP_OR: return ina || inb;
        case OP_ANDNOT: return ina && !inb;
        default: return ina != inb;
    }
}

// ------------------------------------------------------------ tile passes

__device__ __forceinline__ void t_zero(uint64_t *T, uint32_t lane) {
    ulonglong2 *T2 = reinterpret_cast<ulonglong2 *>(T);
#pragma unroll
    for (int k = 0; k < 16; k++) T2[32 * k + lane] = make_ulonglong2(0ull, 0ull);
}

__device__ __forceinline__ void t_load_bitset(uint64_t *T, const uint64_t *g, uint32_t lane) {
    const ulonglong2 *G = reinterpret_cast<const ulonglong2 *>(g);
    ulonglong2 *T2 = reinterpret_cast<ulonglong2 *>(T);
    ulonglong2 v[16];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __ldg(G + 32 * k + lane);
#pragma unroll
    for (int k = 0; k < 16; k++) T2[32 * k + lane] = v[k];
}

// set the bits of an array container (Sec. 3.2: setting the bits at the
// indexes held by an array) into a zeroed tile
__device__ __forceinline__ void t_or_array(uint64_t *T, const uint16_t *v, uint32_t c, uint32_t lane) {
    uint32_t *T32 = reinterpret_cast<uint32_t *>(T);
    for (uint32_t i = lane; i < c; i += 32) {
        uint32_t x = __ldg(v + i);
        atomicOr(T32 + (x >> 5), 1u << (x & 31));
    }
}

// inclusive prefix XOR of the bits of a word, from bit 0 upward
__device__ __forceinline__ uint64_t pxor64(uint64_t x) {
    x ^= x << 1;
    x ^= x << 2;
    x ^= x << 4;
    x ^= x << 8;
    x ^= x << 16;
    x ^= x << 32;
    return x;
}

// expand a run container: toggle bit s and bit e+1 of every run [s, e], then
// a prefix XOR over the 65536-bit string turns the toggles into the runs
static __device__ __noinline__ void t_from_runs(uint64_t *T, const uint32_t *runs, uint32_t r, uint32_t lane) {
    t_zero(T, lane);
    __syncwarp();
    uint32_t *T32 = reinterpret_cast<uint32_t *>(T);
    for (uint32_t i = lane; i < r; i += 32) {
        uint32_t w = __ldg(runs + i);
        uint32_t s = w & 0xFFFFu, e = s + (w >> 16);
        atomicXor(T32 + (s >> 5), 1u << (s & 31));
        if (e < 65535u) {
            uint32_t e1 = e + 1;
            atomicXor(T32 + (e1 >> 5), 1u << (e1 & 31));
        }
    }
    __syncwarp();
    ulonglong2 *T2 = reinterpret_cast<ulonglong2 *>(T);
    uint32_t carry = 0;
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        ulonglong2 w = T2[32 * k + lane];
        uint32_t p0 = __popcll(w.x) & 1u;
        uint32_t pl = (p0 + (uint32_t)__popcll(w.y)) & 1u;
        uint64_t x0 = pxor64(w.x), x1 = pxor64(w.y);
        if (p0) x1 = ~x1;
        uint32_t incl = warp_xor_incl(pl, lane);
        if ((incl ^ pl) ^ carry) {
            x0 = ~x0;
            x1 = ~x1;
        }
        T2[32 * k + lane] = make_ulonglong2(x0, x1);
        carry ^= __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
}

static __device__ __noinline__ void t_decode(uint64_t *T, const CRef &c, uint32_t lane) {
    if (c.type == T_BITSET) {
        t_load_bitset(T, reinterpret_cast<const uint64_t *>(c.p), lane);
    } else if (c.type == T_ARRAY) {
        t_zero(T, lane);
        __syncwarp();
        t_or_array(T, reinterpret_cast<const uint16_t *>(c.p), c.card, lane);
    } else {
        t_from_runs(T, reinterpret_cast<const uint32_t *>(c.p), c.runs, lane);
    }
    __syncwarp();
}

// dst = a op b word by word (a, b: shared tiles or global bitsets), counting
// the result's cardinality c and its number of maximal runs r (a run starts
// at every set bit whose predecessor bit is clear)
template <bool STORE>
__device__ __forceinline__ void t_combine(uint64_t *dst, const uint64_t *a, const uint64_t *b, uint32_t op,
                                          uint32_t &c, uint32_t &r, uint32_t lane) {
    const ulonglong2 *A2 = reinterpret_cast<const ulonglong2 *>(a);
    const ulonglong2 *B2 = reinterpret_cast<const ulonglong2 *>(b);
    ulonglong2 *D2 = reinterpret_cast<ulonglong2 *>(dst);
    uint32_t cc = 0, rr = 0, carry = 0;
    const OpMasks M = op_masks(op);
#pragma unroll 4
    for (int k = 0; k < 16; k++) {
        ulonglong2 x = A2[32 * k + lane], y = B2[32 * k + lane];
        uint64_t z0 = apply_masks(M, x.x, y.x), z1 = apply_masks(M, x.y, y.y);
        if (STORE) D2[32 * k + lane] = make_ulonglong2(z0, z1);
        cc += __popcll(z0) + __popcll(z1);
        uint32_t top = (uint32_t)(z1 >> 63);
        uint32_t prev = __shfl_up_sync(FULL, top, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(FULL, top, 31);
        rr += __popcll(z0 & ~((z0 << 1) | (uint64_t)prev)) + __popcll(z1 & ~((z1 << 1) | (z0 >> 63)));
    }
    c = warp_sum(cc);
    r = warp_sum(rr);
}

// array container from a tile (Sec. 3.1: extract the positions of the set
// bits word by word; here each lane extracts its words and a warp scan of
// the per-lane counts places them)
static __device__ __noinline__ void t_emit_array(const uint64_t *T, uint16_t *out, uint32_t lane) {
    const ulonglong2 *T2 = reinterpret_cast<const ulonglong2 *>(T);
    uint32_t base = 0;
    for (int k = 0; k < 16; k++) {
        ulonglong2 w = T2[32 * k + lane];
        uint32_t n = __popcll(w.x) + __popcll(w.y);
        uint32_t incl = warp_incl(n, lane);
        uint32_t pos = base + incl - n;
        base += __shfl_sync(FULL, incl, 31);
        uint32_t v0 = (uint32_t)(64 * k + 2 * lane) * 64u;
        uint64_t x = w.x;
        while (x) {
            out[pos++] = (uint16_t)(v0 + __ffsll((long long)x) - 1);
            x &= x - 1;
        }
        x = w.y;
        while (x) {
            out[pos++] = (uint16_t)(v0 + 64 + __ffsll((long long)x) - 1);
            x &= x - 1;
        }
    }
}

// run container from a tile: run starts (set bit, clear predecessor) go to
// S, run ends (clear bit after a set one, minus one) to E, both in order;
// then each run is written as start | (length - 1) << 16
static __device__ __noinline__ void t_emit_runs(const uint64_t *T, uint16_t *S, uint16_t *E, uint32_t *out, uint32_t r,
                            uint32_t lane) {
    const ulonglong2 *T2 = reinterpret_cast<const ulonglong2 *>(T);
    uint32_t bs = 0, be = 0, carry = 0;
    for (int k = 0; k < 16; k++) {
        ulonglong2 w = T2[32 * k + lane];
        uint32_t top = (uint32_t)(w.y >> 63);
        uint32_t prev = __shfl_up_sync(FULL, top, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(FULL, top, 31);
        uint64_t sh0 = (w.x << 1) | (uint64_t)prev, sh1 = (w.y << 1) | (w.x >> 63);
        uint64_t st0 = w.x & ~sh0, st1 = w.y & ~sh1;
        uint64_t gs0 = ~w.x & sh0, gs1 = ~w.y & sh1;
        uint32_t ns = __popcll(st0) + __popcll(st1), ne = __popcll(gs0) + __popcll(gs1);
        uint32_t is = warp_incl(ns, lane), ie = warp_incl(ne, lane);
        uint32_t ps = bs + is - ns, pe = be + ie - ne;
        bs += __shfl_sync(FULL, is, 31);
        be += __shfl_sync(FULL, ie, 31);
        uint32_t v0 = (uint32_t)(64 * k + 2 * lane) * 64u;
        while (st0) { S[ps++] = (uint16_t)(v0 + __ffsll((long long)st0) - 1); st0 &= st0 - 1; }
        while (st1) { S[ps++] = (uint16_t)(v0 + 64 + __ffsll((long long)st1) - 1); st1 &= st1 - 1; }
        while (gs0) { E[pe++] = (uint16_t)(v0 + __ffsll((long long)gs0) - 2); gs0 &= gs0 - 1; }
        while (gs1) { E[pe++] = (uint16_t)(v0 + 64 + __ffsll((long long)gs1) - 2); gs1 &= gs1 - 1; }
    }
    if (carry && lane == 0) E[be] = 65535;   // the last run reaches the end of the chunk
    __syncwarp();
    for (uint32_t i = lane; i < r; i += 32) out[i] = (uint32_t)S[i] | ((uint32_t)(E[i] - S[i]) << 16);
}

__device__ __forceinline__ void t_emit_bitset(const uint64_t *T, uint64_t *out, uint32_t lane) {
    const ulonglong2 *T2 = reinterpret_cast<const ulonglong2 *>(T);
    ulonglong2 *O2 = reinterpret_cast<ulonglong2 *>(out);
#pragma unroll
    for (int k = 0; k < 16; k++) O2[32 * k + lane] = T2[32 * k + lane];
}

// ------------------------------------------------------------ probe lists

// keep the values v of array X whose bit in `words` equals `want` (Sec. 3.2
// bit tests; AND keeps present values, ANDNOT absent ones), in order, into L
template <bool STORE>
__device__ uint32_t probe_list(const uint16_t *xv, uint32_t cx, const uint64_t *words, uint32_t want,
                               uint16_t *L, uint32_t lane) {
    uint32_t base = 0;
    for (uint32_t i0 = 0; i0 < cx; i0 += 32) {
        uint32_t i = i0 + lane, v = 0, keep = 0;
        if (i < cx) {
            v = __ldg(xv + i);
            keep = (uint32_t)((words[v >> 6] >> (v & 63)) & 1ull) == want;
        }
        uint32_t m = __ballot_sync(FULL, keep);
        if (STORE && keep) L[base + __popc(m & lanemask_lt(lane))] = (uint16_t)v;
        base += __popc(m);
    }
    __syncwarp();
    return base;
}

__device__ __forceinline__ uint32_t list_runs(const uint16_t *L, uint32_t c, uint32_t lane) {
    uint32_t rr = 0;
    for (uint32_t j = lane; j < c; j += 32) rr += (j == 0 || (uint32_t)L[j] != (uint32_t)L[j - 1] + 1);
    return warp_sum(rr);
}

__device__ __forceinline__ void l_emit_array(const uint16_t *L, uint32_t c, uint16_t *out, uint32_t lane) {
    for (uint32_t j = lane; j < c; j += 32) out[j] = L[j];
}

// runs of a sorted list: compact the indexes of run starts into SI, then run
// k spans L[SI[k]] .. L[SI[k+1] - 1]
static __device__ __noinline__ void l_emit_runs(const uint16_t *L, uint32_t c, uint32_t r, uint16_t *SI, uint32_t *out,
                            uint32_t lane) {
    uint32_t base = 0;
    for (uint32_t j0 = 0; j0 < c; j0 += 32) {
        uint32_t j = j0 + lane;
        uint32_t st = j < c && (j == 0 || (uint32_t)L[j] != (uint32_t)L[j - 1] + 1);
        uint32_t m = __ballot_sync(FULL, st);
        if (st) SI[base + __popc(m & lanemask_lt(lane))] = (uint16_t)j;
        base += __popc(m);
    }
    __syncwarp();
    for (uint32_t k = lane; k < r; k += 32) {
        uint32_t s = SI[k], e = (k + 1 < r ? (uint32_t)SI[k + 1] : c) - 1;
        out[k] = (uint32_t)L[s] | ((uint32_t)(L[e] - L[s]) << 16);
    }
}

// ------------------------------------------------------------ lane sweeps

// interval view of a small container: an array is the intervals [v, v], a
// run container its runs; bounds are half-open [lo, hi)
struct IvSrc {
    const uint8_t *p;
    uint32_t type, n;
};
__device__ __forceinline__ IvSrc iv_src(const CRef &c) {
    IvSrc s;
    s.p = c.p;
    s.type = c.type;
    s.n = c.type == T_ARRAY ? c.card : c.runs;
    return s;
}
__device__ __forceinline__ void iv_at(const IvSrc &s, uint32_t i, uint32_t &lo, uint32_t &hi) {
    if (s.type == T_ARRAY) {
        uint32_t v = __ldg(reinterpret_cast<const uint16_t *>(s.p) + i);
        lo = v;
        hi = v + 1;
    } else {
        uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(s.p) + i);
        lo = w & 0xFFFFu;
        hi = lo + (w >> 16) + 1;
    }
}

// One lane sweeps the boundaries of both interval lists in order and tracks
// membership in A, in B and in the result; result intervals are maximal
// because adjacent input intervals cancel at a shared boundary.  Counts the
// result's cardinality c and runs r; with EMIT it also writes the result as
// an array (u16 values) or as runs (u32 start | (length - 1) << 16).
template <bool EMIT>
__device__ __noinline__ void lane_sweep(uint32_t op, const IvSrc &A, const IvSrc &B, uint32_t &c, uint32_t &r,
                           uint32_t out_type, uint8_t *out) {
    const uint32_t INF = 0x20000u;
    uint32_t ia = 0, ib = 0, aLo = 0, aHi = 0, bLo = 0, bHi = 0;
    uint32_t nxA = INF, nxB = INF;
    bool inA = false, inB = false, inR = false;
    if (A.n) { iv_at(A, 0, aLo, aHi); nxA = aLo; }
    if (B.n) { iv_at(B, 0, bLo, bHi); nxB = bLo; }
    uint32_t rs = 0;
    c = 0;
    r = 0;
    for (;;) {
        uint32_t x = nxA < nxB ? nxA : nxB;
        if (x == INF) break;
        while (nxA == x) {
            if (!inA) { inA = true; nxA = aHi; }
            else {
                inA = false;
                if (++ia < A.n) { iv_at(A, ia, aLo, aHi); nxA = aLo; }
                else nxA = INF;
            }
        }
        while (nxB == x) {
            if (!inB) { inB = true; nxB = bHi; }
            else {
                inB = false;
                if (++ib < B.n) { iv_at(B, ib, bLo, bHi); nxB = bLo; }
                else nxB = INF;
            }
        }
        bool f = member(op, inA, inB);
        if (f != inR) {
            if (f) {
                rs = x;
            } else {
                uint32_t len = x - rs;
                if (EMIT) {
                    if (out_type == T_ARRAY) {
                        uint16_t *o = reinterpret_cast<uint16_t *>(out) + c;
                        for (uint32_t v = 0; v < len; v++) o[v] = (uint16_t)(rs + v);
                    } else {
                        reinterpret_cast<uint32_t *>(out)[r] = rs | ((len - 1) << 16);
                    }
                }
                c += len;
                r++;
            }
            inR = f;
        }
    }
}

}  // namespace rbd
