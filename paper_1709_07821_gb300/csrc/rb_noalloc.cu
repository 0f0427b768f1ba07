// rb_noalloc.cu - decode a bitmap into caller-provided device memory without
// allocating any device memory.
//
// Some callers cannot allocate: their device memory is entirely reserved by
// another allocator (a fixed arena they manage themselves), or they run on a
// path that must never allocate or free (a real-time loop, a callback that
// must not block on an allocator).  For them rb_to_u32_noalloc keeps the one
// piece of scratch the decode needs, the per-container output offsets, in a
// fixed file-scope device array instead of a fresh allocation.
#include <cuda.h>   // driver types only: the two driver calls below are looked up at run time

#include <mutex>

#include "rb_internal.h"

namespace {

constexpr uint32_t NOALLOC_MAX_CONTAINERS = 16384;   // 128 KB of offsets

// Per-container output offsets of every allocation-free decode.  Each device
// that loads the library holds one copy until the process exits; every call
// on that device shares it, so calls whose work overlaps on the device race.
// The scan kernel writes every entry a call reads, so nothing needs clearing.
static __device__ __align__(256) unsigned long long g_noalloc_offs[NOALLOC_MAX_CONTAINERS];

constexpr int MAX_DEVICES = 256;
std::mutex g_mu;
// per device: the device address of g_noalloc_offs and the id of the CUDA
// context it was looked up in.  cudaDeviceReset destroys that context and the
// module is loaded again, possibly at another address, in the next one; a
// call that finds another context id looks the address up again.
void *g_offs_addr[MAX_DEVICES];
unsigned long long g_offs_ctx[MAX_DEVICES];

// cuCtxGetCurrent and cuCtxGetId, from the driver through the runtime (the
// library does not link the driver library itself)
typedef CUresult (*ctx_current_fn)(CUcontext *);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);
ctx_current_fn g_ctx_current;
ctx_id_fn g_ctx_id;

// id of the calling thread's current context (0 if none); g_mu held
bool current_ctx_id(unsigned long long *id) {
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return false;
        g_ctx_current = reinterpret_cast<ctx_current_fn>(f1);
        g_ctx_id = reinterpret_cast<ctx_id_fn>(f2);
    }
    CUcontext c = nullptr;
    if (g_ctx_current(&c) != CUDA_SUCCESS) return false;
    *id = 0;
    return !c || g_ctx_id(c, id) == CUDA_SUCCESS;
}

}  // namespace

extern "C" rb_status rb_to_u32_noalloc(const rb_t *b, uint32_t *dst, uint64_t cap, uint64_t *n_out, void *stream) {
    using namespace rbi;
    clear_stale_error();
    if (!b) return set_err(RB_EINVAL, "rb_to_u32_noalloc: NULL handle");
    if (n_out) *n_out = b->card;
    if (b->n > NOALLOC_MAX_CONTAINERS)
        return set_err(RB_ERANGE, "rb_to_u32_noalloc: the bitmap has %u containers; the allocation-free decode "
                                  "handles at most %u (use rb_to_u32)",
                       b->n, NOALLOC_MAX_CONTAINERS);
    if (b->card == 0) return RB_OK;
    if (!dst) return set_err(RB_EINVAL, "rb_to_u32_noalloc: dst is NULL");
    if (cap < b->card)
        return set_err(RB_ERANGE, "rb_to_u32_noalloc: capacity %llu below cardinality %llu", (unsigned long long)cap,
                       (unsigned long long)b->card);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "rb_to_u32_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return set_err(RB_ERANGE, "rb_to_u32_noalloc: device %d out of range", dev);
    void *offs = nullptr;
    {
        // set-up, once per device (and again after a cudaDeviceReset), with
        // that device current: in host code the array's name is only a
        // stand-in, so kernels get its device address
        std::lock_guard<std::mutex> g(g_mu);
        unsigned long long ctx = 0;
        if (!current_ctx_id(&ctx)) return set_err(RB_ECUDA, "rb_to_u32_noalloc: no current CUDA context id");
        if (!g_offs_addr[dev] || !ctx || g_offs_ctx[dev] != ctx) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_offs);
            if (e != cudaSuccess) return cuda_err(e, "rb_to_u32_noalloc: cudaGetSymbolAddress");
            if (!ctx && !current_ctx_id(&ctx)) return set_err(RB_ECUDA, "rb_to_u32_noalloc: no current CUDA context id");
            g_offs_addr[dev] = p;
            g_offs_ctx[dev] = ctx;
        }
        offs = g_offs_addr[dev];
    }
    e = enqueue_decode(b, reinterpret_cast<uint64_t *>(offs), dst, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(e, "rb_to_u32_noalloc: launch");
    return RB_OK;
}
