// rb_query.cu - membership queries and the cosine similarity.
//
// Membership follows Sec. 1 of the paper: the value's 16 most significant
// bits select a container by binary search over the sorted keys, and the 16
// least significant bits are then looked up in that container (a bit test in
// a bitset, a binary search in an array or in the runs).  One thread answers
// one value; the values of a batch are independent.
#include "rb_device.cuh"

using namespace rbi;
using namespace rbd;

namespace {

// is the low half v in the container described by d (payload at p)?
__device__ __forceinline__ uint8_t container_has(const uint8_t *p, uint64_t d, uint32_t v) {
    const uint32_t t = d_type(d);
    if (t == T_BITSET) {
        const uint64_t w = __ldg(reinterpret_cast<const unsigned long long *>(p) + (v >> 6));
        return (uint8_t)((w >> (v & 63)) & 1ull);
    }
    if (t == T_ARRAY) {
        const uint16_t *a = reinterpret_cast<const uint16_t *>(p);
        uint32_t lo = 0, hi = d_card(d);
        while (lo < hi) {
            const uint32_t m = (lo + hi) >> 1;
            if ((uint32_t)__ldg(a + m) < v) lo = m + 1;
            else hi = m;
        }
        return (uint8_t)(lo < d_card(d) && (uint32_t)__ldg(a + lo) == v);
    }
    // runs: the last run starting at or before v must reach it
    const uint32_t *r = reinterpret_cast<const uint32_t *>(p);
    uint32_t lo = 0, hi = d_runs(d);
    while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if ((__ldg(r + m) & 0xFFFFu) <= v) lo = m + 1;
        else hi = m;
    }
    if (lo == 0) return 0;
    const uint32_t w = __ldg(r + lo - 1), s = w & 0xFFFFu;
    return (uint8_t)(v - s <= (w >> 16));
}

__global__ void k_contains(const uint16_t *__restrict__ keys, const uint64_t *__restrict__ descs, const uint8_t *base,
                           uint32_t n, const uint32_t *__restrict__ vals, uint64_t nv, uint8_t *__restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nv; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = __ldg(vals + i), key = x >> 16;
        const uint32_t j = lower_bound16(keys, n, key);
        uint8_t r = 0;
        if (j < n && (uint32_t)__ldg(keys + j) == key) {
            const uint64_t d = __ldg(descs + j);
            r = container_has(base + d_off(d), d, x & 0xFFFFu);
        }
        out[i] = r;
    }
}

}  // namespace

extern "C" {

rb_status rb_contains_many(const rb_t *b, const uint32_t *vals, uint64_t n, int on_device, uint8_t *out,
                           void *stream) {
    clear_stale_error();
    if (!b) return set_err(RB_EINVAL, "rb_contains_many: NULL handle");
    if (n == 0) return RB_OK;
    if (!vals || !out) return set_err(RB_EINVAL, "rb_contains_many: NULL vals or out");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t *dv = vals;
    uint8_t *dout = out;
    uint8_t *tmp = nullptr;
    const uint64_t vbytes = align_up(4 * n, 256), tbytes = vbytes + align_up(n, 256);
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        tmp = (uint8_t *)dev_alloc(tbytes, s);
        if (!tmp) return RB_ENOMEM;
        dv = (const uint32_t *)tmp;
        dout = tmp + vbytes;
        e = cudaMemcpyAsync(tmp, vals, 4 * n, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        const uint64_t need = (n + 255) / 256, cap = (uint64_t)sm_count() * 16;
        k_contains<<<(unsigned)(need < cap ? need : cap), 256, 0, s>>>(b->keys, b->descs, b->base, b->n, dv, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(out, dout, n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(s);
    if (tmp) dev_free(tmp, tbytes, s);
    if (e != cudaSuccess) return cuda_err(e, "rb_contains_many");
    return RB_OK;
}

rb_status rb_contains(const rb_t *b, uint32_t value, int *out) {
    if (!out) return set_err(RB_EINVAL, "rb_contains: out is NULL");
    uint8_t r = 0;
    rb_status st = rb_contains_many(b, &value, 1, 0, &r, nullptr);
    if (st == RB_OK) *out = r;
    return st;
}

rb_status rb_cosine(const rb_t *a, const rb_t *b, double *out, uint64_t *inter, void *stream) {
    if (!a || !b) return set_err(RB_EINVAL, "rb_cosine: NULL handle");
    uint64_t i = 0;
    rb_status st = rb_and_cardinality(a, b, &i, stream);
    if (st != RB_OK) return st;
    if (inter) *inter = i;
    if (out) *out = (a->card && b->card) ? (double)i / sqrt((double)a->card * (double)b->card) : 0.0;
    return RB_OK;
}

}  // extern "C"
