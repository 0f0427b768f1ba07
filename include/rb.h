/*
 * rb.h - C ABI of the GB300 (sm_103a) Roaring bitmap library.
 *
 * A Roaring bitmap stores a set of 32-bit integers as a sorted list of 16-bit
 * keys (the high halves present in the set), each paired with one container
 * holding the low halves of that chunk: a bitset of 2^16 bits, an array of at
 * most 4096 sorted values, or a list of runs <s,l> meaning [s, s+l]
 * (arXiv 1709.07821, Sec. 1, Fig. 1).  Every bitmap this library hands out is
 * in canonical form: no empty container, and each container of cardinality c
 * with r maximal runs is a run container iff (c <= 4096 and 2r < c) or
 * (c > 4096 and r <= 2047), else an array iff c <= 4096, else a bitset
 * (Sec. 1's type constraints, read as "smallest of array 2c B, bitset 8 KB,
 * runs 4r B").
 *
 * Conventions for every entry point:
 *  - Bitmaps live in device memory of the current CUDA device; rb_t is an
 *    opaque host handle.  Inputs are never modified (Sec. 5: operations build
 *    a new bitmap and leave their inputs unchanged).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that return host-visible results (counts, new handles) synchronise that
 *    stream before returning.
 *  - Every rb_t** output is a new handle owned by the caller and released
 *    with rb_free().  On error *out is set to NULL and nothing leaks.
 *  - Errors: each call returns an rb_status; rb_last_error() gives a message
 *    for the calling thread's last failure.
 *  - Device memory comes from the allocator installed with
 *    rb_set_allocator() (default: cudaMallocAsync / cudaFreeAsync).
 */
#ifndef RB_H
#define RB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rb rb_t;

typedef enum {
    RB_OK = 0,
    RB_EINVAL = 1,    /* bad argument: NULL handle, unsorted input, bad op ... */
    RB_ENOMEM = 2,    /* the allocator returned NULL */
    RB_ECUDA = 3,     /* a CUDA runtime call failed (message has the reason) */
    RB_ETIMEOUT = 4,  /* a bounded wait ran out */
    RB_EBUSY = 5,     /* admission refused: not enough budget right now */
    RB_ERANGE = 6     /* a size exceeds a documented limit */
} rb_status;

/* Sec. 1: intersection = AND, union = OR, difference = ANDNOT,
 * symmetric difference = XOR. */
typedef enum { RB_AND = 0, RB_OR = 1, RB_ANDNOT = 2, RB_XOR = 3 } rb_op;

/* container type codes used by rb_export_layout */
enum { RB_TYPE_ARRAY = 0, RB_TYPE_BITSET = 1, RB_TYPE_RUN = 2 };

/* ---------------------------------------------------------------- memory */

/* Device allocator hooks.  alloc returns a device pointer (16-byte aligned at
 * least) or NULL; release gets back the pointer and size it was given.  The
 * stream is the one the memory is first used on.  Passing NULL for both
 * restores the default (cudaMallocAsync / cudaFreeAsync). */
typedef void *(*rb_alloc_fn)(uint64_t bytes, void *stream, void *ctx);
typedef void (*rb_free_fn)(void *ptr, uint64_t bytes, void *stream, void *ctx);
rb_status rb_set_allocator(rb_alloc_fn alloc, rb_free_fn release, void *ctx);

/* --------------------------------------------------------- construction */

/* Build a bitmap from n strictly increasing uint32 values (Sec. 1: chunk by
 * the high 16 bits, keep the low 16 bits in the chunk's container, type
 * chosen by the canonical rule).  `vals` is a device pointer if
 * vals_on_device != 0, else host memory (copied in on `stream`).  Unsorted or
 * duplicate input returns RB_EINVAL.  n == 0 gives the empty bitmap. */
rb_status rb_from_sorted_u32(const uint32_t *vals, uint64_t n, int vals_on_device, void *stream,
                             rb_t **out);

/* Write the set's values in ascending order to dst (device memory if
 * dst_on_device != 0, else host memory), at most cap of them; *n_out gets the
 * cardinality.  cap < cardinality returns RB_ERANGE and writes nothing. */
rb_status rb_to_u32(const rb_t *b, uint32_t *dst, int dst_on_device, uint64_t cap, uint64_t *n_out,
                    void *stream);

/* Cardinality (sum of container cardinalities; Sec. 5 "Fast counts"). */
rb_status rb_cardinality(const rb_t *b, uint64_t *out);

/* Number of containers and the size of the exported payload (array 2c B,
 * bitset 8192 B, run 4r B per container). */
rb_status rb_info(const rb_t *b, uint32_t *n_containers, uint64_t *payload_bytes);

/* Copy the canonical layout to host arrays: keys[n] (u16), types[n] (u8,
 * RB_TYPE_*), cards[n] (u32), offs[n + 1] (u64, byte offsets into payload),
 * and payload (array: ascending u16; bitset: 1024 little-endian u64 words,
 * bit v & 63 of word v >> 6; runs: (start, length - 1) u16 pairs, Sec. 1 and
 * Fig. 1).  payload_cap below the size from rb_info returns RB_ERANGE. */
rb_status rb_export_layout(const rb_t *b, uint16_t *keys, uint8_t *types, uint32_t *cards,
                           uint64_t *offs, uint8_t *payload, uint64_t payload_cap, void *stream);

/* Release a handle (NULL is ignored).  Device memory shared with other
 * handles of the same batch is returned when its last handle is freed. */
void rb_free(rb_t *b);

/* rb_free on each of hs[0..n) (NULL entries are ignored), e.g. all results
 * of a batch at once. */
void rb_free_array(rb_t *const *hs, uint64_t n);

/* ------------------------------------------------------------- pairwise */

/* out = a op b as a new canonical bitmap (Sec. 1 set operations; Sec. 5
 * materialised pairwise operations).  Key merge, per-container-pair work and
 * canonical compaction all run on the device. */
rb_status rb_apply(rb_op op, const rb_t *a, const rb_t *b, rb_t **out, void *stream);
rb_status rb_and(const rb_t *a, const rb_t *b, rb_t **out, void *stream);
rb_status rb_or(const rb_t *a, const rb_t *b, rb_t **out, void *stream);
rb_status rb_andnot(const rb_t *a, const rb_t *b, rb_t **out, void *stream);
rb_status rb_xor(const rb_t *a, const rb_t *b, rb_t **out, void *stream);

/* |a op b| without materialising the result.  Sec. 5 "Fast counts": only
 * |a n b| is computed on the device; |a u b| = |a| + |b| - |a n b|,
 * |a \ b| = |a| - |a n b|, |a xor b| = |a| + |b| - 2 |a n b|. */
rb_status rb_apply_cardinality(rb_op op, const rb_t *a, const rb_t *b, uint64_t *out, void *stream);
rb_status rb_and_cardinality(const rb_t *a, const rb_t *b, uint64_t *out, void *stream);
rb_status rb_or_cardinality(const rb_t *a, const rb_t *b, uint64_t *out, void *stream);
rb_status rb_andnot_cardinality(const rb_t *a, const rb_t *b, uint64_t *out, void *stream);
rb_status rb_xor_cardinality(const rb_t *a, const rb_t *b, uint64_t *out, void *stream);

/* Jaccard index |a n b| / |a u b| (Sec. 5 "Fast counts").  inter and uni
 * (either may be NULL) receive the two integers; *out is their quotient as a
 * correctly rounded double, and 0.0 when both sets are empty. */
rb_status rb_jaccard(const rb_t *a, const rb_t *b, double *out, uint64_t *inter, uint64_t *uni,
                     void *stream);

/* Cosine similarity |a n b| / sqrt(|a| |b|) (Sec. 5 "Fast counts" names it
 * beside the Jaccard index).  |a n b| is counted on the device; *out is
 * (double)|a n b| / sqrt((double)|a| * (double)|b|) with IEEE double
 * operations, and 0.0 when either set is empty.  inter (may be NULL)
 * receives |a n b|. */
rb_status rb_cosine(const rb_t *a, const rb_t *b, double *out, uint64_t *inter, void *stream);

/* -------------------------------------------------------- serialisation */

/* A portable byte image of one bitmap, for snapshots of a resident index
 * (Sec. 5 notes that Roaring has a portable serialized form but does not
 * give it; this format is the library's own).  Little endian:
 *   u32 magic 0x42474252, u32 version 1, u32 n (containers), u32 0,
 *   u64 cardinality, u64 payload bytes,
 *   u16 keys[n] (strictly increasing), u16 runs[n] (run containers: number
 *   of runs, else 0), u8 types[n] (RB_TYPE_*), zero bytes to a multiple of
 *   4, u32 cards[n], then every container's payload in key order exactly as
 *   rb_export_layout writes it.
 * rb_serialize: *n_bytes (may be NULL) gets the image size; with buf NULL
 * nothing else happens, else the image is written to buf (host memory, cap
 * bytes; RB_ERANGE if smaller).  Synchronises `stream`. */
rb_status rb_serialize(const rb_t *b, uint8_t *buf, uint64_t cap, uint64_t *n_bytes, void *stream);
/* A new bitmap from an image (host memory, len bytes).  Every field is
 * checked on the host first (sizes, key order, sorted and maximal values
 * and runs, cardinalities, the canonical type of each container); anything
 * else returns RB_EINVAL and allocates nothing.  One upload on `stream`,
 * synchronised before returning. */
rb_status rb_deserialize(const uint8_t *buf, uint64_t len, void *stream, rb_t **out);

/* ----------------------------------------------------------- membership */

/* Membership of n values (Sec. 1: binary search over the 16-bit keys, then
 * a bit test in a bitset or a search in an array or run container).
 * out[i] = 1 if vals[i] is in b, else 0.  With on_device != 0, vals (n
 * uint32) and out (n bytes) are device memory and the call only enqueues the
 * work on `stream`; otherwise both are host memory, copied in and out, and
 * the stream is synchronised.  n == 0 does nothing. */
rb_status rb_contains_many(const rb_t *b, const uint32_t *vals, uint64_t n, int on_device, uint8_t *out,
                           void *stream);
/* One value: *out = 1 if value is in b, else 0 (synchronous, default stream). */
rb_status rb_contains(const rb_t *b, uint32_t value, int *out);

/* -------------------------------------------------------------- batches */

/* One query of a batch: op (rb_op), indexes a and b into the pool, flags. */
typedef struct {
    uint32_t op;
    uint32_t a;
    uint32_t b;
    uint32_t flags;
} rb_query;
#define RB_Q_COUNT_ONLY 1u   /* return |a op b| only; no bitmap */

/* Run nq pairwise queries over a pool of bitmaps in one persistent,
 * work-stealing launch over container pairs (no paper counterpart: the
 * batching pattern of this library).  outs[i] receives the result bitmap of a
 * materialising query and NULL for a count-only one (outs may be NULL when
 * every query is count-only); counts[i] (counts may be NULL) receives the
 * result's cardinality.  Results are identical to nq separate rb_apply /
 * rb_apply_cardinality calls.  Preparing a batch of 16,384 or more
 * queries (here and in rb_plan_create) spreads its per-query host passes
 * over up to 8 short-lived threads, joined before the call returns. */
rb_status rb_batch_op(const rb_t *const *pool, uint32_t pool_n, const rb_query *q, uint64_t nq,
                      rb_t **outs, uint64_t *counts, void *stream);

/* Jaccard indexes of n pairs (a[i], b[i]) of the pool, count-only. */
rb_status rb_batch_jaccard(const rb_t *const *pool, uint32_t pool_n, const uint32_t *a,
                           const uint32_t *b, uint64_t n, double *jac, uint64_t *inter,
                           uint64_t *uni, void *stream);

/* A reusable batch: the host-side preparation (key counts, slot and tile
 * prefix sums, device tables) is done once; each rb_plan_run replays the
 * launch sequence as a CUDA graph and returns fresh result handles.  The
 * pool's bitmaps must outlive the plan. */
typedef struct rb_plan rb_plan_t;
rb_status rb_plan_create(const rb_t *const *pool, uint32_t pool_n, const rb_query *q, uint64_t nq,
                         void *stream, rb_plan_t **out);
rb_status rb_plan_run(rb_plan_t *p, rb_t **outs, uint64_t *counts, void *stream);
/* rb_plan_run in two halves, so that the host can prepare or consume other
 * work while the device runs: rb_plan_launch enqueues a run (a graph replay
 * on the plan's own stream, ordered after the work already on `stream`, and
 * `stream` ordered after it) and returns at once; rb_plan_collect waits for
 * it, reruns it with exact sizes if its output space ran out, and fills outs
 * and counts as rb_plan_run does.  One run per plan may be outstanding
 * (RB_EINVAL otherwise, and for a collect without a launch); rb_plan_run and
 * rb_autotune on a plan with an outstanding run return RB_EINVAL; several
 * plans launched on one stream run one after another on the device. */
rb_status rb_plan_launch(rb_plan_t *p, void *stream);
rb_status rb_plan_collect(rb_plan_t *p, rb_t **outs, uint64_t *counts);
/* Measurements of the last run, from CUDA events on the stream the kernels
 * ran on: the container-pair stage is a lean kernel (key merge, copies of
 * unmatched containers), a small-pair kernel (the array pairs and small run
 * pairs the lean one queued) and a heavy kernel (pairs with a bitset, many
 * values or many runs, and bitset copies).  *_bytes are the algorithmic
 * bytes of each kernel's share of the work: the input payloads the op must
 * read (AND: matched containers; OR, XOR: every container; ANDNOT: all of
 * a, matched of b) and the output payloads, counted by the kernels
 * themselves, plus 15 bytes of key and metadata per container of both
 * inputs (lean kernel) and per output container, and 8 bytes per
 * count-only result; deferred and small_pairs are the numbers of pairs
 * queued for the heavy and the small-pair kernel. */
typedef struct {
    double lean_ms, heavy_ms;
    uint64_t lean_bytes, heavy_bytes, alg_bytes, out_bytes, deferred;
    double small_ms;
    uint64_t small_bytes, small_pairs;
} rb_plan_timing;
rb_status rb_plan_stats(const rb_plan_t *p, rb_plan_timing *t);
void rb_plan_free(rb_plan_t *p);

/* ------------------------------------------------------------ schedules */

/* Launch schedule of the container-pair kernels: the heavy kernel's warps
 * per CTA (2, 4 or 8; each warp owns 16 KB of shared tiles) and CTAs per SM;
 * the largest array pair (values on both sides) that one lane of the
 * small-pair kernel merges alone (larger array pairs up to 254 values are
 * merged by groups of 8 lanes, up to 1022 by the whole warp; bitsets and
 * larger containers are deferred to the heavy kernel); the lean kernel's
 * CTAs of 128 threads per SM (0 = 8, the most that fit); how many 128-byte
 * lines of each queued container's payload the lean kernel hints into L2
 * ahead of use (0 = none); and how many consecutive 32-slot tiles a lean
 * kernel warp takes from the shared work counter at once (1 .. 256; 0 =
 * 32; plans too small to give every warp about 64 takes of that size take
 * fewer).  The multi-way kernel (rb_multi_op and the serving loop) takes
 * warps_per_cta from here and runs as many CTAs per SM as fit. */
typedef struct {
    uint32_t warps_per_cta;
    uint32_t ctas_per_sm;
    uint32_t small_intervals;
    uint32_t lean_ctas_per_sm;
    uint32_t prefetch_lines;
    uint32_t tiles_per_take;
} rb_schedule;
rb_status rb_set_schedule(const rb_schedule *s);
rb_status rb_get_schedule(rb_schedule *s);

/* Tune the schedule on the plan (no paper counterpart): coordinate descent
 * from the current schedule over the heavy kernel's shape ({2,6}, {4,3},
 * {8,1} warps per CTA x CTAs per SM), small_intervals (32, 48, 64, 96, 128),
 * lean_ctas_per_sm (6, 7, 8), prefetch_lines (0, 2, 4, 8) and
 * tiles_per_take (8, 16, 32, 64): each pass
 * times every value of one knob with the others fixed (one warm-up run,
 * then reps runs, CUDA events on `stream`, key merge + container-pair
 * kernels) and keeps the fastest, until a pass changes nothing (at most 3
 * passes).  The fastest is installed as the current schedule and returned
 * in *best with its time in *best_ms.  Results do not depend on the
 * schedule. */
rb_status rb_autotune(rb_plan_t *p, uint32_t reps, void *stream, rb_schedule *best,
                      double *best_ms);

/* ------------------------------------------------------------ multi-way */

/* out = in[0] op in[1] op ... op in[k-1] for op RB_AND or RB_OR (Sec. 5 "Wide
 * unions": the union of many sets; the intersection likewise), computed key
 * by key in one pass: each output key folds its k containers once.  card (may
 * be NULL) receives the result's cardinality.  out may be NULL for a
 * count-only evaluation.  k == 0 gives the empty set. */
rb_status rb_multi_op(rb_op op, const rb_t *const *in, uint32_t k, rb_t **out, uint64_t *card,
                      void *stream);

/* --------------------------------------------------------- accumulation */

/* In-place accumulation acc = acc op b over a stream of bitmaps, op RB_OR or
 * RB_AND (Sec. 5 "Wide unions": a union of many bitmaps computed partly in
 * place; Sec. 2.2: lazy operations that skip the cardinality of
 * intermediate results).  The accumulator holds one 8 KB bitset tile per
 * key present; creation reserves a 65536-entry key map and max_keys tiles
 * (max_keys * 8 KB + 2 MB of device memory, from the installed allocator),
 * and no later call allocates device memory except rb_accum_result's
 * output.  rb_accum_add only enqueues work on `stream` (OR: each of b's
 * containers is OR-ed into its key's tile, touching only the words it
 * covers; AND: the first add fills the accumulator, later ones drop the keys
 * b lacks and AND the rest).  Calls on one accumulator must be ordered (one
 * stream, or synchronised).  If the keys added exceed max_keys, the adds
 * skip the keys that find no tile and rb_accum_result returns RB_ERANGE.
 * rb_accum_result canonicalises the current state into a new bitmap (out,
 * may be NULL for the cardinality only) without changing the accumulator,
 * and synchronises `stream`.  rb_accum_reset empties it. */
typedef struct rb_accum rb_accum_t;
rb_status rb_accum_create(rb_op op, uint32_t max_keys, void *stream, rb_accum_t **out);
rb_status rb_accum_add(rb_accum_t *acc, const rb_t *b, void *stream);
rb_status rb_accum_result(rb_accum_t *acc, rb_t **out, uint64_t *card, void *stream);
rb_status rb_accum_reset(rb_accum_t *acc, void *stream);
void rb_accum_free(rb_accum_t *acc);

/* -------------------------------------------------------------- serving */

/* A serving loop over a device-resident index (no paper counterpart).
 * Requests are multi-way AND / OR queries over index members, materialised
 * or count-only.  A host thread admits queued requests in arrival order
 * while a stream slot is free (max_inflight_batches) and the memory budget
 * covers each request's worst-case result bytes, batches them (at most
 * max_batch per batch), and launches each batch on its own stream, so
 * batches overlap on the device while new requests keep arriving
 * (continuous batching).  Result memory is charged to mem_budget until the
 * caller frees the result; the loop allocates it (and each batch's tables)
 * with cudaMallocAsync from its own thread, not through the installed
 * allocator, whose hooks may have to run on the caller's thread (a Python
 * allocator needs the interpreter lock).  The index table is allocated by
 * rb_server_create through the installed allocator.  rb_server_destroy
 * completes batches in flight and fails requests never admitted with
 * RB_EBUSY. */
#define RB_SERVE_MAX_K 8
typedef struct {
    uint32_t op;            /* RB_AND or RB_OR */
    uint32_t k;             /* 1 .. RB_SERVE_MAX_K members */
    uint32_t count_only;    /* non-zero: cardinality only */
    uint32_t members[RB_SERVE_MAX_K];
} rb_request;

typedef struct rb_server rb_server_t;
rb_status rb_server_create(const rb_t *const *index, uint32_t n, uint64_t mem_budget,
                           uint32_t max_inflight_batches, uint32_t max_batch,
                           rb_server_t **out);
/* Queue a request; returns at once with a ticket.  RB_EBUSY if the request
 * alone exceeds the whole budget. */
rb_status rb_server_submit(rb_server_t *s, const rb_request *r, uint64_t *ticket);
/* Wait (at most timeout_ms) for a ticket.  *out (may be NULL) receives the
 * result bitmap of a materialising request (caller frees it); *card its
 * cardinality; *latency_s the time from submit to completion on the device.
 * RB_ETIMEOUT if it is not done in time (the ticket stays valid); RB_EINVAL
 * for an unknown ticket, or one that rb_server_poll collected meanwhile.
 * Safe to call from several threads while others submit and poll. */
rb_status rb_server_wait(rb_server_t *s, uint64_t ticket, int timeout_ms, rb_t **out,
                         uint64_t *card, double *latency_s);
/* Queue n requests at once (a frontend draining its input in bursts): the
 * same checks as rb_server_submit for every request, then all are queued
 * with one lock and the same submit time; tickets[i] is request i's ticket.
 * On a bad request nothing is queued and its error is returned. */
rb_status rb_server_submit_many(rb_server_t *s, const rb_request *r, uint32_t n, uint64_t *tickets);
/* Collect up to cap completed requests in completion order, waiting at most
 * timeout_ms for the first one; *n_out gets how many (0 on timeout).  For
 * each: tickets[i], status[i] (RB_OK or the request's error), outs[i] (the
 * result bitmap of a materialising request, owned by the caller; NULL
 * otherwise; with outs == NULL every result is freed at once), cards[i],
 * latency_s[i] (submit to completion on the device).  status, outs, cards
 * and latency_s may be NULL.  A collected ticket is no longer valid. */
rb_status rb_server_poll(rb_server_t *s, uint32_t cap, int timeout_ms, uint64_t *tickets, rb_status *status,
                         rb_t **outs, uint64_t *cards, double *latency_s, uint32_t *n_out);
/* Counters: completed requests, launched batches, peak requests in flight. */
rb_status rb_server_stats(rb_server_t *s, uint64_t *completed, uint64_t *batches,
                          uint64_t *peak_inflight);
void rb_server_destroy(rb_server_t *s);

/* ------------------------------------------------------ allocation-free */

/* rb_to_u32 for callers that cannot allocate device memory: code whose
 * device memory is wholly reserved by another allocator, or paths that must
 * never allocate or free (real-time loops, callbacks that must not block).
 * The paper has no counterpart.  Writes the set's values in ascending order
 * to dst (DEVICE memory owned by the caller, cap values at most) and *n_out
 * (may be NULL) gets the cardinality.  It allocates nothing: the decode's
 * per-container offsets live in a fixed device array of 16384 entries
 * (128 KB, one per device that loads the library, kept until the process
 * exits), so a bitmap with more than 16384 containers returns RB_ERANGE, as
 * does cap below the cardinality.  Every call on a device shares that array:
 * calls whose work overlaps on the device race.  The first call on each
 * device looks up the array's device address (set-up, with that device
 * current); make that first call before any stream capture.  After a
 * cudaDeviceReset the array may be reloaded elsewhere: the next call on that
 * device sees the new context and repeats the set-up.  The call only
 * enqueues work on `stream`: the values are in dst once the stream reaches
 * it.  RB_ECUDA if a CUDA call fails. */
rb_status rb_to_u32_noalloc(const rb_t *b, uint32_t *dst, uint64_t cap, uint64_t *n_out, void *stream);

/* ----------------------------------------------------------------- misc */

/* Self-test of the bounded-wait error path; the paper has no counterpart.
 * Every spin-wait in the library's kernels (the bulk-copy barriers of the
 * heavy kernel) gives up after a cycle limit, records the timeout in a
 * status word and returns, so that the host reports RB_ETIMEOUT and the
 * context stays usable.  This call runs one warp that waits on a
 * shared-memory barrier expecting two arrivals, with limit_cycles (1..2^31
 * SM cycles) as the limit: with complete != 0 both arrivals happen and it
 * returns RB_OK; with complete == 0 only one does, the wait runs out and it
 * returns RB_ETIMEOUT.  Synchronises `stream`.  RB_EINVAL for a limit out of
 * range, RB_ENOMEM / RB_ECUDA as elsewhere. */
rb_status rb_selftest_wait(uint64_t limit_cycles, int complete, void *stream);

/* Message describing the calling thread's last error ("" if none). */
const char *rb_last_error(void);

/* Library version string. */
const char *rb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RB_H */
