// rb_internal.h - internal structures of the GB300 Roaring library.
//
// Device layout of one bitmap (structure of arrays, all in one allocation):
//   keys  u16[n]   sorted high halves (Sec. 1: one entry per non-empty chunk)
//   descs u64[n]   packed container descriptor, one 8-byte load per container:
//                    bits  0..15  cardinality - 1       (1 .. 65536)
//                    bits 16..17  type: 0 array, 1 bitset, 2 runs (Sec. 2.2: one
//                                 type tag per container instead of tagged pointers)
//                    bits 18..28  number of runs (run containers; else 0; <= 2047)
//                    bits 29..63  payload offset / 4 from the bitmap's base (128 GiB reach)
//   payload        arrays: u16 values, allocation rounded up to 4 bytes;
//                  runs: u32 per run = start | (length - 1) << 16;
//                  bitsets: 1024 u64 words, 16-byte aligned.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>

#include "rb.h"

namespace rbi {

constexpr uint32_t T_ARRAY = 0, T_BITSET = 1, T_RUN = 2, T_NONE = 3;
constexpr uint64_t DESC_EMPTY = ~0ull;           // type field 3: "no container"
constexpr uint64_t MAX_OFFSET = (1ull << 37);    // 35-bit offset in 4-byte units
constexpr uint32_t ARRAY_MAX = 4096;             // Sec. 1
constexpr uint32_t RUN_MAX_LARGE = 2047;         // Sec. 1

__host__ __device__ __forceinline__ uint64_t mk_desc(uint32_t card, uint32_t type, uint32_t runs,
                                                     uint64_t off_bytes) {
    return (uint64_t)(card - 1) | ((uint64_t)type << 16) | ((uint64_t)runs << 18) |
           ((off_bytes >> 2) << 29);
}
__host__ __device__ __forceinline__ uint32_t d_card(uint64_t d) { return (uint32_t)(d & 0xFFFFu) + 1; }
__host__ __device__ __forceinline__ uint32_t d_type(uint64_t d) { return (uint32_t)(d >> 16) & 3u; }
__host__ __device__ __forceinline__ uint32_t d_runs(uint64_t d) { return (uint32_t)(d >> 18) & 0x7FFu; }
__host__ __device__ __forceinline__ uint64_t d_off(uint64_t d) { return (d >> 29) << 2; }

// canonical container type (Sec. 1 constraints read as minimum memory;
// strict inequalities decide ties)
__host__ __device__ __forceinline__ uint32_t canon_type(uint32_t c, uint32_t r) {
    if (c <= ARRAY_MAX) return (2 * r < c) ? T_RUN : T_ARRAY;
    return (r <= RUN_MAX_LARGE) ? T_RUN : T_BITSET;
}
// payload bytes as exported (array 2c, bitset 8192, runs 4r)
__host__ __device__ __forceinline__ uint32_t payload_bytes(uint32_t type, uint32_t c, uint32_t r) {
    return type == T_ARRAY ? 2 * c : type == T_BITSET ? 8192u : 4 * r;
}
// bytes reserved in a word region (arrays rounded up to 4 bytes)
__host__ __device__ __forceinline__ uint32_t word_alloc_bytes(uint32_t type, uint32_t c, uint32_t r) {
    return type == T_ARRAY ? ((2 * c + 3) & ~3u) : 4 * r;
}

// device view of one bitmap (32 bytes)
struct BmView {
    const uint16_t *keys;
    const uint64_t *descs;
    const uint8_t *base;
    uint32_t n;
    uint32_t pad;
};

}  // namespace rbi

// ------------------------------------------------------------------ host side

#include <mutex>

// memory budget shared by a serving loop and the result arenas it hands out;
// it lives until the loop and every arena charged to it are gone.  notify
// (the loop's wake-up, with the loop as ctx) is called and cleared under mu,
// so that no call is in progress once the loop has cleared it
struct RbBudget {
    std::atomic<int64_t> used;
    std::atomic<int> refs;
    std::mutex mu;
    void (*notify)(void *ctx);
    void *ctx;
};

// reference-counted device allocation shared by the handles of one batch
struct RbArena {
    void *ptr;
    uint64_t bytes;
    cudaStream_t stream;
    std::atomic<int> refs;
    int native;            // 1: cudaMallocAsync, regardless of the installed hooks
    RbBudget *budget;      // charged `charge` bytes until released (may be NULL)
    uint64_t charge;
};

struct RbBlock;

struct rb {
    uint32_t n;            // containers
    uint64_t card;         // total cardinality
    uint64_t word_bytes;   // bytes of array/run payload (allocation sizes)
    uint32_t n_bitsets;    // bitset containers
    uint16_t *keys;        // device
    uint64_t *descs;       // device
    uint8_t *base;         // device: descriptor offsets are relative to this
    RbArena *arena;        // owner of keys/descs/payload memory (may be shared)
    RbBlock *block;        // handles of one batch are allocated together (NULL: alone)
};

// the handles of one batch's results, allocated as one array and released
// when the last of them is freed
struct RbBlock {
    std::atomic<uint64_t> refs;
    rb *items;
};

namespace rbi {

// errors
rb_status set_err(rb_status st, const char *fmt, ...);
rb_status cuda_err(cudaError_t e, const char *what);
#define RB_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return ::rbi::cuda_err(_e, #call);      \
    } while (0)

// allocator
void *dev_alloc(uint64_t bytes, cudaStream_t s);
void dev_free(void *p, uint64_t bytes, cudaStream_t s);
RbArena *arena_new(uint64_t bytes, cudaStream_t s);   // NULL on failure (error set)
RbArena *arena_new_native(uint64_t bytes, cudaStream_t s);
void *dev_alloc_native(uint64_t bytes, cudaStream_t s);
void dev_free_native(void *p, cudaStream_t s);
void budget_unref(RbBudget *b);
void arena_ref(RbArena *a);
void arena_unref(RbArena *a);
void arena_unref_n(RbArena *a, int n);   // n references at once

// pinned host staging buffer of the calling thread (grows; never shrinks)
void *pinned_scratch(uint64_t bytes);

int sm_count();
inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }
// drop a stale, non-sticky error left by an earlier tolerated call, so that
// the launch checks of this call report only its own failures
inline void clear_stale_error() { (void)cudaGetLastError(); }

BmView view_of(const rb *b);
rb *handle_new();

// decode kernels of rb_to_u32 with caller-provided offsets scratch (b->n > 0)
cudaError_t enqueue_decode(const rb *b, uint64_t *offs, uint32_t *out, cudaStream_t s);

// shared launch schedule
rb_schedule current_schedule();

}  // namespace rbi
