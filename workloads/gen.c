/*
 * gen.c - seeded synthetic set generator for the Roaring workloads.
 *
 * This module holds no Roaring arithmetic: it only draws sorted, distinct
 * uint32 values (the input every bitmap is built from) and query lists.  Both
 * the CPU oracle and the CUDA library ingest exactly these arrays.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014; the finaliser constants are the published
 * ones).  Each bitmap draws from its own stream keyed by (seed, bitmap index),
 * so generation is parallel and reproducible.  All sampling is integer-only,
 * except the log-uniform cardinality law, which uses det_exp() below: plain
 * IEEE double +,*,/ (compiled with -ffp-contract=off), so x86-64 and aarch64
 * produce the same bits.
 *
 * Shapes follow the paper's datasets (Sec. 5 "Data", Table 2: 200 sets per
 * collection, universes 2e5..4.3e6, densities 0.0008..0.17; sorted variants
 * are run-heavy) and the five workload recipes of the build.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct { uint64_t s; } rng_t;

static inline uint64_t sm64(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static rng_t make_stream(uint64_t seed, uint64_t idx) {
    rng_t r;
    r.s = seed * 0xD1B54A32D192ED03ull + (idx + 1) * 0x9E3779B97F4A7C15ull;
    (void)sm64(&r);
    r.s ^= sm64(&r);
    return r;
}

/* uniform integer in [0, n), n >= 1 (multiply-shift; bias < n / 2^64) */
static inline uint64_t below(rng_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)sm64(r) * n) >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double unif01(rng_t *r) {
    return (double)(sm64(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* exp(x) by range reduction and a Taylor polynomial; deterministic across
 * platforms because it uses only correctly rounded IEEE operations. */
static double det_exp(double x) {
    const double LN2_HI = 6.93147180369123816490e-01;
    const double LN2_LO = 1.90821492927058770002e-10;
    double kf = x * 1.4426950408889634 + (x >= 0 ? 0.5 : -0.5);
    long k = (long)kf;
    double r = (x - (double)k * LN2_HI) - (double)k * LN2_LO;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 24; i++) { term = term * r / (double)i; sum += term; }
    /* multiply by 2^k exactly */
    while (k > 0) { sum *= 2.0; k--; }
    while (k < 0) { sum *= 0.5; k++; }
    return sum;
}

/* round(10^U(lo, hi)) */
static uint64_t log_uniform(rng_t *r, double lo, double hi) {
    double e = lo + (hi - lo) * unif01(r);
    double v = det_exp(e * 2.302585092994045684);
    uint64_t c = (uint64_t)(v + 0.5);
    return c < 1 ? 1 : c;
}

/* number of Bernoulli(2^-k) trials up to and including the first success:
 * geometric on {1,2,...} with mean 2^k */
static uint32_t geom_pow2(rng_t *r, int k) {
    uint32_t n = 1;
    uint64_t mask = (1ull << k) - 1;
    for (;;) {
        uint64_t w = sm64(r);
        for (int t = 0; t + k <= 64; t += k) {
            if (((w >> t) & mask) == 0) return n;
            n++;
        }
    }
}

/* ---------------- growable u32 vector ---------------- */
typedef struct { uint32_t *v; uint64_t n, cap; } vec_t;

static int vec_reserve(vec_t *a, uint64_t cap) {
    if (cap <= a->cap) return 0;
    uint64_t nc = a->cap ? a->cap : 1024;
    while (nc < cap) nc *= 2;
    uint32_t *p = (uint32_t *)realloc(a->v, nc * sizeof(uint32_t));
    if (!p) return -1;
    a->v = p; a->cap = nc;
    return 0;
}
static inline int vec_push(vec_t *a, uint32_t x) {
    if (a->n == a->cap && vec_reserve(a, a->n + 1)) return -1;
    a->v[a->n++] = x;
    return 0;
}

/* LSD radix sort of u32 by two 16-bit digits */
static int radix_sort_u32(uint32_t *v, uint64_t n) {
    if (n < 2) return 0;
    uint32_t *tmp = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)malloc(65536 * sizeof(uint64_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    for (int pass = 0; pass < 2; pass++) {
        int sh = pass * 16;
        memset(cnt, 0, 65536 * sizeof(uint64_t));
        for (uint64_t i = 0; i < n; i++) cnt[(v[i] >> sh) & 0xFFFF]++;
        uint64_t s = 0;
        for (int d = 0; d < 65536; d++) { uint64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (uint64_t i = 0; i < n; i++) tmp[cnt[(v[i] >> sh) & 0xFFFF]++] = v[i];
        memcpy(v, tmp, n * sizeof(uint32_t));
    }
    free(tmp); free(cnt);
    return 0;
}

/* c distinct uniform values in [0, universe), sorted (c <= universe / 2) */
static int gen_uniform(rng_t *r, uint64_t c, uint64_t universe, vec_t *out) {
    if (c > universe) c = universe;
    if (vec_reserve(out, c)) return -1;
    uint64_t got = 0;
    out->n = 0;
    while (got < c) {
        for (uint64_t i = got; i < c; i++) out->v[i] = (uint32_t)below(r, universe);
        if (radix_sort_u32(out->v, c)) return -1;
        uint64_t w = 0;
        for (uint64_t i = 0; i < c; i++)
            if (w == 0 || out->v[i] != out->v[w - 1]) out->v[w++] = out->v[i];
        got = w;
    }
    out->n = c;
    return 0;
}

/* dense-clustered: from a random start chunk, consecutive 2^16 chunks filled
 * with Bernoulli(d) bits until c values are drawn */
static int gen_dense(rng_t *r, uint64_t c, double d_lo, double d_hi, vec_t *out) {
    double d = d_lo + (d_hi - d_lo) * unif01(r);
    uint64_t thr = (uint64_t)(d * 4294967296.0);
    uint64_t chunks_needed = (uint64_t)((double)c / (65536.0 * d)) + 2;
    if (chunks_needed > 65536) chunks_needed = 65536;
    uint64_t k0 = below(r, 65536 - chunks_needed + 1);
    out->n = 0;
    if (vec_reserve(out, c)) return -1;
    for (uint64_t k = k0; k < 65536 && out->n < c; k++) {
        for (uint32_t b = 0; b < 65536 && out->n < c; b += 2) {
            uint64_t w = sm64(r);
            if ((w & 0xFFFFFFFFull) < thr) out->v[out->n++] = (uint32_t)((k << 16) | b);
            if (out->n < c && (w >> 32) < thr) out->v[out->n++] = (uint32_t)((k << 16) | (b + 1));
        }
    }
    return 0;
}

/* run-heavy: from a random start, alternate runs of Geom(mean 2^run_k) values
 * and gaps of Geom(mean 2^gap_k) missing values, until c values or the end of
 * the universe */
static int gen_runs(rng_t *r, uint64_t c, uint64_t universe, int run_k, int gap_k, vec_t *out) {
    uint64_t span = c * (((uint64_t)1 << gap_k) / ((uint64_t)1 << run_k) + 2);
    uint64_t start = span >= universe ? 0 : below(r, universe - span);
    uint64_t pos = start;
    out->n = 0;
    if (vec_reserve(out, c)) return -1;
    while (out->n < c && pos < universe) {
        uint64_t len = geom_pow2(r, run_k);
        for (uint64_t i = 0; i < len && out->n < c && pos < universe; i++) out->v[out->n++] = (uint32_t)pos++;
        pos += geom_pow2(r, gap_k);
    }
    return 0;
}

/* ---------------- pool generation ---------------- */

typedef struct {
    uint64_t seed;
    uint32_t n_bitmaps;
    uint32_t universe_log2;   /* 24, 26 or 32 */
    double log10_lo, log10_hi;/* cardinality law: round(10^U(lo, hi)) */
    uint32_t pm_sparse, pm_dense, pm_runs; /* class mixture, per mille */
    uint32_t run_k, gap_k;    /* run / gap lengths: Geom with mean 2^k */
    double d_lo, d_hi;        /* density law of the dense-clustered class */
} gen_params;

typedef struct {
    uint32_t n;
    vec_t *sets;
    uint8_t *cls;
} gen_pool;

typedef struct {
    const gen_params *p;
    gen_pool *pool;
    uint32_t next;
    pthread_mutex_t mu;
    int err;
} job_t;

static int gen_one(const gen_params *p, uint32_t i, vec_t *out, uint8_t *cls) {
    rng_t r = make_stream(p->seed, i);
    uint64_t universe = p->universe_log2 >= 32 ? (1ull << 32) : (1ull << p->universe_log2);
    uint64_t c = log_uniform(&r, p->log10_lo, p->log10_hi);
    uint32_t u = (uint32_t)below(&r, 1000);
    if (u < p->pm_sparse) { *cls = 0; return gen_uniform(&r, c, universe, out); }
    if (u < p->pm_sparse + p->pm_dense) { *cls = 1; return gen_dense(&r, c, p->d_lo, p->d_hi, out); }
    *cls = 2;
    return gen_runs(&r, c, universe, (int)p->run_k, (int)p->gap_k, out);
}

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        uint32_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->p->n_bitmaps) break;
        if (gen_one(j->p, i, &j->pool->sets[i], &j->pool->cls[i])) {
            pthread_mutex_lock(&j->mu); j->err = 1; pthread_mutex_unlock(&j->mu);
        }
    }
    return NULL;
}

void gen_pool_free(gen_pool *g) {
    if (!g) return;
    for (uint32_t i = 0; i < g->n; i++) free(g->sets[i].v);
    free(g->sets); free(g->cls); free(g);
}

gen_pool *gen_pool_create(const gen_params *p, int threads) {
    gen_pool *g = (gen_pool *)calloc(1, sizeof(gen_pool));
    if (!g) return NULL;
    g->n = p->n_bitmaps;
    g->sets = (vec_t *)calloc(p->n_bitmaps ? p->n_bitmaps : 1, sizeof(vec_t));
    g->cls = (uint8_t *)calloc(p->n_bitmaps ? p->n_bitmaps : 1, 1);
    if (!g->sets || !g->cls) { gen_pool_free(g); return NULL; }
    job_t j; j.p = p; j.pool = g; j.next = 0; j.err = 0;
    pthread_mutex_init(&j.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < threads; t++)
        if (pthread_create(&th[t], NULL, worker, &j) == 0) started++;
    if (started == 0) worker(&j);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.mu);
    if (j.err) { gen_pool_free(g); return NULL; }
    return g;
}

/* bitmaps idx[0..n) of the pool p describes, as a pool of n sets (set j is
 * bitmap idx[j], with exactly the values gen_pool_create gives it): a large
 * pool can be drawn a slice at a time */
typedef struct {
    const gen_params *p;
    const uint32_t *idx;
    uint32_t n, next;
    gen_pool *pool;
    pthread_mutex_t mu;
    int err;
} some_job_t;

static void *some_worker(void *arg) {
    some_job_t *j = (some_job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        uint32_t t = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (t >= j->n) break;
        if (gen_one(j->p, j->idx[t], &j->pool->sets[t], &j->pool->cls[t])) {
            pthread_mutex_lock(&j->mu); j->err = 1; pthread_mutex_unlock(&j->mu);
        }
    }
    return NULL;
}

gen_pool *gen_pool_create_some(const gen_params *p, const uint32_t *idx, uint32_t n, int threads) {
    gen_pool *g = (gen_pool *)calloc(1, sizeof(gen_pool));
    if (!g) return NULL;
    g->n = n;
    g->sets = (vec_t *)calloc(n ? n : 1, sizeof(vec_t));
    g->cls = (uint8_t *)calloc(n ? n : 1, 1);
    if (!g->sets || !g->cls) { gen_pool_free(g); return NULL; }
    for (uint32_t t = 0; t < n; t++)
        if (idx[t] >= p->n_bitmaps) { gen_pool_free(g); return NULL; }
    some_job_t j; j.p = p; j.idx = idx; j.n = n; j.next = 0; j.pool = g; j.err = 0;
    pthread_mutex_init(&j.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < threads; t++)
        if (pthread_create(&th[t], NULL, some_worker, &j) == 0) started++;
    if (started == 0) some_worker(&j);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.mu);
    if (j.err) { gen_pool_free(g); return NULL; }
    return g;
}

uint32_t gen_pool_n(const gen_pool *g) { return g->n; }
uint64_t gen_pool_size(const gen_pool *g, uint32_t i) { return g->sets[i].n; }
const uint32_t *gen_pool_values(const gen_pool *g, uint32_t i) { return g->sets[i].v; }
uint32_t gen_pool_class(const gen_pool *g, uint32_t i) { return g->cls[i]; }

/* ---------------- the two-bitmap "plain method" workload ----------------
 * 300 distinct keys in [0,1024): the first 100 go to both bitmaps, the next
 * 100 to the first only, the last 100 to the second only.  Per bitmap the
 * keys are shuffled and position i mod 3 picks the kind of chunk: uniform
 * values with c ~ U{1..4096}, uniform values with c ~ U{4097..60000}, or
 * n ~ U{10..200} runs with lengths ~ U{1..500} separated by gaps >= 1. */

static int fill_uniform16(rng_t *r, uint32_t key, uint32_t c, vec_t *out) {
    uint8_t *mark = (uint8_t *)calloc(65536, 1);
    if (!mark) return -1;
    int invert = c > 32768;
    uint32_t want = invert ? 65536 - c : c, got = 0;
    while (got < want) {
        uint32_t v = (uint32_t)below(r, 65536);
        if (!mark[v]) { mark[v] = 1; got++; }
    }
    for (uint32_t v = 0; v < 65536; v++)
        if ((mark[v] != 0) != invert) vec_push(out, (key << 16) | v);
    free(mark);
    return 0;
}

static int fill_runs16(rng_t *r, uint32_t key, vec_t *out) {
    for (;;) {
        uint32_t n = 10 + (uint32_t)below(r, 191);
        uint32_t len[200], total = 0;
        for (uint32_t i = 0; i < n; i++) { len[i] = 1 + (uint32_t)below(r, 500); total += len[i]; }
        if (total + (n - 1) > 65536) continue;
        uint32_t free_space = 65536 - total - (n - 1);
        /* random composition of free_space into n+1 parts via n sorted bars */
        uint32_t bars[200];
        for (uint32_t i = 0; i < n; i++) bars[i] = (uint32_t)below(r, (uint64_t)free_space + 1);
        for (uint32_t i = 1; i < n; i++) {   /* insertion sort, n <= 200 */
            uint32_t x = bars[i]; int k = (int)i - 1;
            while (k >= 0 && bars[k] > x) { bars[k + 1] = bars[k]; k--; }
            bars[k + 1] = x;
        }
        uint32_t pos = bars[0];
        for (uint32_t i = 0; i < n; i++) {
            for (uint32_t t = 0; t < len[i]; t++) vec_push(out, (key << 16) | (pos + t));
            pos += len[i];
            if (i + 1 < n) pos += 1 + (bars[i + 1] - bars[i]);
        }
        return 0;
    }
}

static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : x > y;
}

gen_pool *gen_plain_pair(uint64_t seed) {
    gen_pool *g = (gen_pool *)calloc(1, sizeof(gen_pool));
    if (!g) return NULL;
    g->n = 2;
    g->sets = (vec_t *)calloc(2, sizeof(vec_t));
    g->cls = (uint8_t *)calloc(2, 1);
    rng_t r = make_stream(seed, 0);
    uint32_t perm[1024];
    for (uint32_t i = 0; i < 1024; i++) perm[i] = i;
    for (uint32_t i = 0; i < 300; i++) {
        uint32_t j = i + (uint32_t)below(&r, 1024 - i);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int side = 0; side < 2; side++) {
        uint32_t keys[200];
        for (uint32_t i = 0; i < 100; i++) keys[i] = perm[i];
        for (uint32_t i = 0; i < 100; i++) keys[100 + i] = perm[(side == 0 ? 100 : 200) + i];
        rng_t rs = make_stream(seed, 1 + side);
        for (uint32_t i = 199; i > 0; i--) {
            uint32_t j = (uint32_t)below(&rs, i + 1);
            uint32_t t = keys[i]; keys[i] = keys[j]; keys[j] = t;
        }
        vec_t *out = &g->sets[side];
        for (uint32_t i = 0; i < 200; i++) {
            uint32_t kind = i % 3;
            if (kind == 0) fill_uniform16(&rs, keys[i], 1 + (uint32_t)below(&rs, 4096), out);
            else if (kind == 1) fill_uniform16(&rs, keys[i], 4097 + (uint32_t)below(&rs, 60000 - 4097 + 1), out);
            else fill_runs16(&rs, keys[i], out);
        }
        qsort(out->v, out->n, sizeof(uint32_t), cmp_u32);
    }
    return g;
}

/* ---------------- query lists ---------------- */

/* pairs (a, b), a != b, uniform over the pool; op by per-mille thresholds:
 * u < t0 -> 0 (AND), < t1 -> 1 (OR), < t2 -> 2 (ANDNOT), else 3 (XOR) */
void gen_pairs(uint64_t seed, uint64_t n_pairs, uint32_t pool_n, uint32_t t0, uint32_t t1, uint32_t t2,
               uint32_t *op, uint32_t *a, uint32_t *b) {
    rng_t r = make_stream(seed, 0xFFFFFFFFull);
    for (uint64_t i = 0; i < n_pairs; i++) {
        uint32_t u = (uint32_t)below(&r, 1000);
        op[i] = u < t0 ? 0 : u < t1 ? 1 : u < t2 ? 2 : 3;
        uint32_t x = (uint32_t)below(&r, pool_n);
        uint32_t y = (uint32_t)below(&r, pool_n - 1);
        if (y >= x) y++;
        a[i] = x; b[i] = y;
    }
}

/* multi-way queries: k ~ U{k_lo..k_hi} distinct members, op AND/OR 50/50,
 * count-only 50/50; members written k_hi per query (unused = 0xFFFFFFFF) */
void gen_multi_queries(uint64_t seed, uint64_t nq, uint32_t pool_n, uint32_t k_lo, uint32_t k_hi,
                       uint32_t *op, uint32_t *k, uint32_t *count_only, uint32_t *members) {
    rng_t r = make_stream(seed, 0xFFFFFFFEull);
    for (uint64_t q = 0; q < nq; q++) {
        uint32_t kk = k_lo + (uint32_t)below(&r, k_hi - k_lo + 1);
        op[q] = (uint32_t)below(&r, 2);
        count_only[q] = (uint32_t)below(&r, 2);
        k[q] = kk;
        uint32_t *m = members + q * k_hi;
        for (uint32_t i = 0; i < k_hi; i++) m[i] = 0xFFFFFFFFu;
        for (uint32_t i = 0; i < kk; i++) {
            for (;;) {
                uint32_t x = (uint32_t)below(&r, pool_n);
                int dup = 0;
                for (uint32_t t = 0; t < i; t++) dup |= (m[t] == x);
                if (!dup) { m[i] = x; break; }
            }
        }
    }
}
