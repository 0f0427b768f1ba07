/*
 * oracle.c - plain, slow CPU oracle for Roaring bitmap set operations.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * What it computes (Lemire et al., "Roaring Bitmaps: Implementation of an
 * Optimized Software Library", arXiv 1709.07821):
 *
 *  - Sec. 1: a set of 32-bit integers is split into chunks by the 16 most
 *    significant bits; each non-empty chunk is a container holding the 16
 *    least significant bits, as a bitset (2^16 bits), an array (<= 4096 sorted
 *    values) or runs (sorted pairs <s,l> meaning [s, s+l]).  The container
 *    type is picked to minimise memory; no bitset holds fewer than 4097
 *    values, no array more than 4096, and a run container with more than
 *    4096 values has at most 2047 runs, otherwise fewer runs than half its
 *    values.  Empty containers are omitted (Sec. 2.2).
 *  - Sec. 1: intersection = AND, union = OR, difference = ANDNOT, symmetric
 *    difference = XOR.
 *  - Sec. 5 "Fast counts": Jaccard index |A n B| / |A u B| and cosine
 *    similarity |A n B| / sqrt(|A| |B|).
 *  - Sec. 1 / Sec. 5 "Membership queries": is x in the set?
 *  - Sec. 5 "Wide unions": the union of many sets, computed as a sequential
 *    fold over the inputs.
 *
 * Method: every operation works chunk by chunk.  For each key it decodes the
 * (at most two) containers into sorted lists of 16-bit values, merges the two
 * lists with the operation's membership rule, and re-encodes the result in
 * canonical form (encode() below).  No blocking, vectorisation or type-pair
 * specialisation: a reader can check each step against the definitions.
 *
 * Canonical form (the reading of Sec. 1's type rule used throughout): with c
 * the cardinality of a chunk and r its number of maximal runs of consecutive
 * values, sizes are array 2c bytes, bitset 8192 bytes, runs 4r bytes; the
 * chunk is a run container iff (c <= 4096 and 2r < c) or (c > 4096 and
 * r <= 2047); otherwise an array iff c <= 4096; otherwise a bitset.
 * Payloads: array = ascending u16; bitset = 1024 little-endian u64 words, bit
 * (v & 63) of word (v >> 6); runs = (start, length - 1) u16 pairs ascending.
 *
 * Export format (the parity interface): per container key u16, type u8
 * (0 array, 1 bitset, 2 runs), card u32, and its payload bytes concatenated
 * in key order with offsets u64[n + 1].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_ARRAY = 0, O_BITSET = 1, O_RUN = 2 };
enum { O_AND = 0, O_OR = 1, O_ANDNOT = 2, O_XOR = 3 };
enum { O_OK = 0, O_EINVAL = 1, O_ENOMEM = 2 };

typedef struct {
    uint16_t key;
    uint8_t type;
    uint32_t card;
    uint32_t nbytes;
    uint8_t *data;
} ocont;

typedef struct {
    uint32_t n;
    ocont *c;
} obm;

/* number of maximal runs of consecutive values in a sorted distinct list */
static uint32_t count_runs(const uint16_t *v, uint32_t c) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < c; i++)
        if (i == 0 || (uint32_t)v[i] != (uint32_t)v[i - 1] + 1) r++;
    return r;
}

/* Sec. 1 type rule, read as "smallest of array 2c B, bitset 8 KB, runs 4r B",
 * with the paper's strict inequalities deciding ties */
static uint8_t choose_type(uint32_t c, uint32_t r) {
    if (c <= 4096) return (2 * r < c) ? O_RUN : O_ARRAY;
    return (r <= 2047) ? O_RUN : O_BITSET;
}

/* canonical container for a non-empty sorted distinct list of low halves */
static int encode(uint16_t key, const uint16_t *v, uint32_t c, ocont *out) {
    uint32_t r = count_runs(v, c);
    out->key = key;
    out->card = c;
    out->type = choose_type(c, r);
    if (out->type == O_ARRAY) {
        out->nbytes = 2 * c;
        out->data = (uint8_t *)malloc(out->nbytes);
        if (!out->data) return O_ENOMEM;
        for (uint32_t i = 0; i < c; i++) {
            out->data[2 * i] = (uint8_t)(v[i] & 0xFF);
            out->data[2 * i + 1] = (uint8_t)(v[i] >> 8);
        }
    } else if (out->type == O_BITSET) {
        out->nbytes = 8192;
        out->data = (uint8_t *)calloc(8192, 1);
        if (!out->data) return O_ENOMEM;
        /* bit v lives in byte v/8, bit v%8 (same as u64 word v>>6, bit v&63
         * in little-endian order) */
        for (uint32_t i = 0; i < c; i++) out->data[v[i] >> 3] |= (uint8_t)(1u << (v[i] & 7));
    } else {
        out->nbytes = 4 * r;
        out->data = (uint8_t *)malloc(out->nbytes);
        if (!out->data) return O_ENOMEM;
        uint32_t k = 0, i = 0;
        while (i < c) {
            uint32_t j = i;
            while (j + 1 < c && (uint32_t)v[j + 1] == (uint32_t)v[j] + 1) j++;
            uint16_t s = v[i], l = (uint16_t)(v[j] - v[i]);
            out->data[4 * k + 0] = (uint8_t)(s & 0xFF);
            out->data[4 * k + 1] = (uint8_t)(s >> 8);
            out->data[4 * k + 2] = (uint8_t)(l & 0xFF);
            out->data[4 * k + 3] = (uint8_t)(l >> 8);
            k++;
            i = j + 1;
        }
    }
    return O_OK;
}

/* sorted list of low halves held by a container; returns its length */
static uint32_t decode(const ocont *x, uint16_t *out) {
    uint32_t n = 0;
    if (x->type == O_ARRAY) {
        for (uint32_t i = 0; i < x->card; i++)
            out[n++] = (uint16_t)(x->data[2 * i] | (x->data[2 * i + 1] << 8));
    } else if (x->type == O_BITSET) {
        for (uint32_t v = 0; v < 65536; v++)
            if (x->data[v >> 3] & (1u << (v & 7))) out[n++] = (uint16_t)v;
    } else {
        for (uint32_t k = 0; k < x->nbytes / 4; k++) {
            uint32_t s = x->data[4 * k] | (x->data[4 * k + 1] << 8);
            uint32_t l = x->data[4 * k + 2] | (x->data[4 * k + 3] << 8);
            for (uint32_t v = s; v <= s + l; v++) out[n++] = (uint16_t)v;
        }
    }
    return n;
}

/* merge two sorted distinct lists by the operation's membership rule
 * (Sec. 1: AND keeps values in both, OR in either, ANDNOT in the first only,
 * XOR in exactly one) */
static uint32_t merge_lists(int op, const uint16_t *a, uint32_t na, const uint16_t *b, uint32_t nb,
                            uint16_t *out) {
    uint32_t i = 0, j = 0, n = 0;
    while (i < na || j < nb) {
        int in_a, in_b;
        uint16_t v;
        if (j == nb || (i < na && a[i] < b[j])) { v = a[i++]; in_a = 1; in_b = 0; }
        else if (i == na || b[j] < a[i]) { v = b[j++]; in_a = 0; in_b = 1; }
        else { v = a[i]; i++; j++; in_a = 1; in_b = 1; }
        int keep = 0;
        switch (op) {
            case O_AND: keep = in_a && in_b; break;
            case O_OR: keep = in_a || in_b; break;
            case O_ANDNOT: keep = in_a && !in_b; break;
            case O_XOR: keep = in_a != in_b; break;
        }
        if (keep && out) out[n] = v;
        n += (uint32_t)keep;
    }
    return n;
}

void orc_free(obm *b) {
    if (!b) return;
    for (uint32_t i = 0; i < b->n; i++) free(b->c[i].data);
    free(b->c);
    free(b);
}

static obm *new_bm(uint32_t cap) {
    obm *b = (obm *)calloc(1, sizeof(obm));
    if (!b) return NULL;
    b->c = (ocont *)calloc(cap ? cap : 1, sizeof(ocont));
    if (!b->c) { free(b); return NULL; }
    return b;
}

/* Build from a strictly increasing uint32 list (Sec. 1: chunk by the high
 * 16 bits, store the low 16 bits).  Unsorted or duplicate input is rejected
 * with O_EINVAL. */
obm *orc_from_sorted_u32(const uint32_t *v, uint64_t n, int *status) {
    *status = O_OK;
    for (uint64_t i = 1; i < n; i++)
        if (v[i] <= v[i - 1]) { *status = O_EINVAL; return NULL; }
    uint32_t nkeys = 0;
    for (uint64_t i = 0; i < n; i++)
        if (i == 0 || (v[i] >> 16) != (v[i - 1] >> 16)) nkeys++;
    obm *b = new_bm(nkeys);
    uint16_t *low = (uint16_t *)malloc(65536 * sizeof(uint16_t));
    if (!b || !low) { orc_free(b); free(low); *status = O_ENOMEM; return NULL; }
    uint64_t i = 0;
    while (i < n) {
        uint32_t key = v[i] >> 16, c = 0;
        while (i < n && (v[i] >> 16) == key) low[c++] = (uint16_t)(v[i++] & 0xFFFF);
        if (encode((uint16_t)key, low, c, &b->c[b->n])) { orc_free(b); free(low); *status = O_ENOMEM; return NULL; }
        b->n++;
    }
    free(low);
    return b;
}

/* A op B as a new canonical bitmap; the inputs are unchanged (Sec. 5). */
obm *orc_op(int op, const obm *a, const obm *b) {
    obm *r = new_bm(a->n + b->n);
    uint16_t *la = (uint16_t *)malloc(65536 * 2), *lb = (uint16_t *)malloc(65536 * 2);
    uint16_t *lr = (uint16_t *)malloc(65536 * 2);
    if (!r || !la || !lb || !lr) { orc_free(r); free(la); free(lb); free(lr); return NULL; }
    uint32_t i = 0, j = 0;
    while (i < a->n || j < b->n) {
        uint32_t ka = i < a->n ? a->c[i].key : 0x10000u;
        uint32_t kb = j < b->n ? b->c[j].key : 0x10000u;
        uint32_t key = ka < kb ? ka : kb;
        uint32_t na = 0, nb = 0;
        if (ka == key) na = decode(&a->c[i++], la);
        if (kb == key) nb = decode(&b->c[j++], lb);
        uint32_t nr = merge_lists(op, la, na, lb, nb, lr);
        if (nr) {
            if (encode((uint16_t)key, lr, nr, &r->c[r->n])) { orc_free(r); r = NULL; break; }
            r->n++;
        }
    }
    free(la); free(lb); free(lr);
    return r;
}

/* |A op B| counted directly from the merged lists (no materialisation) */
uint64_t orc_op_card(int op, const obm *a, const obm *b) {
    uint16_t *la = (uint16_t *)malloc(65536 * 2), *lb = (uint16_t *)malloc(65536 * 2);
    uint64_t total = 0;
    if (!la || !lb) { free(la); free(lb); return (uint64_t)-1; }
    uint32_t i = 0, j = 0;
    while (i < a->n || j < b->n) {
        uint32_t ka = i < a->n ? a->c[i].key : 0x10000u;
        uint32_t kb = j < b->n ? b->c[j].key : 0x10000u;
        uint32_t key = ka < kb ? ka : kb;
        uint32_t na = 0, nb = 0;
        if (ka == key) na = decode(&a->c[i++], la);
        if (kb == key) nb = decode(&b->c[j++], lb);
        total += merge_lists(op, la, na, lb, nb, NULL);
    }
    free(la); free(lb);
    return total;
}

uint64_t orc_card(const obm *b) {
    uint64_t s = 0;
    for (uint32_t i = 0; i < b->n; i++) s += b->c[i].card;
    return s;
}

/* Jaccard index |A n B| / |A u B| (Sec. 5 "Fast counts"); both sets empty
 * gives 0 with inter = uni = 0. */
double orc_jaccard(const obm *a, const obm *b, uint64_t *inter, uint64_t *uni) {
    *inter = orc_op_card(O_AND, a, b);
    *uni = orc_op_card(O_OR, a, b);
    return *uni ? (double)*inter / (double)*uni : 0.0;
}

/* Cosine similarity |A n B| / sqrt(|A| |B|) (Sec. 5 "Fast counts"), in IEEE
 * double arithmetic; 0 when either set is empty. */
double orc_cosine(const obm *a, const obm *b, uint64_t *inter) {
    *inter = orc_op_card(O_AND, a, b);
    uint64_t ca = orc_card(a), cb = orc_card(b);
    if (ca == 0 || cb == 0) return 0.0;
    return (double)*inter / sqrt((double)ca * (double)cb);
}

/* Membership of each value (Sec. 1): the chunk of the value's high 16 bits,
 * then its low 16 bits within that chunk's container.  Plain scans: the
 * containers in order, an array's values in order, each run in turn. */
void orc_contains(const obm *b, const uint32_t *v, uint64_t n, uint8_t *out) {
    for (uint64_t i = 0; i < n; i++) {
        uint32_t key = v[i] >> 16, low = v[i] & 0xFFFF;
        uint8_t r = 0;
        for (uint32_t c = 0; c < b->n; c++) {
            const ocont *x = &b->c[c];
            if (x->key != key) continue;
            if (x->type == O_BITSET) {
                r = (x->data[low >> 3] >> (low & 7)) & 1;
            } else if (x->type == O_ARRAY) {
                for (uint32_t k = 0; k < x->card && !r; k++)
                    r = (uint32_t)(x->data[2 * k] | (x->data[2 * k + 1] << 8)) == low;
            } else {
                for (uint32_t k = 0; k < x->nbytes / 4 && !r; k++) {
                    uint32_t s = x->data[4 * k] | (x->data[4 * k + 1] << 8);
                    uint32_t l = x->data[4 * k + 2] | (x->data[4 * k + 3] << 8);
                    r = low >= s && low <= s + l;
                }
            }
            break;
        }
        out[i] = r;
    }
}

static obm *copy_bm(const obm *a) {
    obm *r = new_bm(a->n);
    if (!r) return NULL;
    for (uint32_t i = 0; i < a->n; i++) {
        r->c[i] = a->c[i];
        r->c[i].data = (uint8_t *)malloc(a->c[i].nbytes ? a->c[i].nbytes : 1);
        if (!r->c[i].data) { r->n = i; orc_free(r); return NULL; }
        memcpy(r->c[i].data, a->c[i].data, a->c[i].nbytes);
    }
    r->n = a->n;
    return r;
}

/* op over k inputs as the sequential fold acc = acc op S_i (Sec. 5 "Wide
 * unions" proceeds this way); k == 0 gives the empty set. */
obm *orc_multi(int op, const obm *const *in, uint32_t k) {
    if (k == 0) return new_bm(0);
    obm *acc = copy_bm(in[0]);
    for (uint32_t i = 1; i < k && acc; i++) {
        obm *nx = orc_op(op, acc, in[i]);
        orc_free(acc);
        acc = nx;
    }
    return acc;
}

uint32_t orc_n(const obm *b) { return b->n; }

uint64_t orc_payload_bytes(const obm *b) {
    uint64_t s = 0;
    for (uint32_t i = 0; i < b->n; i++) s += b->c[i].nbytes;
    return s;
}

/* values in ascending order; returns how many were written (<= cap) */
uint64_t orc_to_u32(const obm *b, uint32_t *out, uint64_t cap) {
    uint16_t *l = (uint16_t *)malloc(65536 * 2);
    uint64_t n = 0;
    if (!l) return 0;
    for (uint32_t i = 0; i < b->n; i++) {
        uint32_t m = decode(&b->c[i], l);
        for (uint32_t t = 0; t < m && n < cap; t++) out[n++] = ((uint32_t)b->c[i].key << 16) | l[t];
    }
    free(l);
    return n;
}

void orc_export(const obm *b, uint16_t *keys, uint8_t *types, uint32_t *cards, uint64_t *offs,
                uint8_t *payload) {
    uint64_t o = 0;
    for (uint32_t i = 0; i < b->n; i++) {
        keys[i] = b->c[i].key;
        types[i] = b->c[i].type;
        cards[i] = b->c[i].card;
        offs[i] = o;
        memcpy(payload + o, b->c[i].data, b->c[i].nbytes);
        o += b->c[i].nbytes;
    }
    offs[b->n] = o;
}
