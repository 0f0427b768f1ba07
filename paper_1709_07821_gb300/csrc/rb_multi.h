// rb_multi.h - internal interface of the multi-way engine (k-way AND / OR),
// shared by rb_multi_op and the serving loop.
#pragma once

#include <vector>

#include "rb_internal.h"

namespace rbi {

struct MultiQuery {
    uint32_t op;          // RB_AND or RB_OR
    uint32_t count_only;
    std::vector<uint32_t> members;   // indexes into the pool
};

struct MultiBatch;   // opaque

// reusable pinned staging memory for the host side of a batch
struct PinnedBuf {
    uint8_t *p = nullptr;
    uint64_t cap = 0;
};

// upper bound on the device bytes one query's results can take (metadata,
// word payload and bitsets), the same bound multi_prepare sizes arenas with
uint64_t multi_query_bound(const rb *const *pool, const MultiQuery &q);

// Host-side preparation of a batch over a pool whose device views are
// d_pool (pool_n entries) and whose host handles are pool[].  Computes the
// slot/tile layout and an upper bound on the result bytes (arena_bytes) that
// no run can exceed.  The device tables are allocated here (on stream s).
// `stage` (may be NULL) is reused for the pinned host mirrors; `native`
// selects cudaMallocAsync for the device tables (used from the serving thread).
rb_status multi_prepare(const rb *const *pool, const BmView *d_pool, uint32_t pool_n,
                        const std::vector<MultiQuery> &qs, cudaStream_t s, MultiBatch **out,
                        uint64_t *arena_bytes, PinnedBuf *stage = nullptr, bool native = false);
// Enqueue the launch sequence on s, writing results into `arena` (at least
// arena_bytes; may be NULL when every query is count-only).  No host sync.
rb_status multi_enqueue(MultiBatch *b, RbArena *arena, cudaStream_t s);
// After the stream work completed: fill result handles (outs[i] NULL for
// count-only queries) and cardinalities.  Handles take a reference on arena.
rb_status multi_finish(MultiBatch *b, RbArena *arena, rb_t **outs, uint64_t *cards);
void multi_free(MultiBatch *b, cudaStream_t s);

}  // namespace rbi
