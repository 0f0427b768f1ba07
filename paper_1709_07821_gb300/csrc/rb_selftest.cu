// rb_selftest.cu - exercises the bounded-wait error path that every
// spin-wait of the library's kernels takes (a shared-memory barrier whose
// phase does not complete within a cycle limit), without faulting anything:
// the waiting kernel records the timeout in a status word and returns.
#include "rb_device.cuh"

using namespace rbi;
using namespace rbd;

namespace {

// One warp.  The barrier expects two arrivals; lane 0 always arrives, lane 1
// only when `complete` is set.  Lane 0 then waits on the phase with the
// given cycle limit and stores 1 (completed) or 2 (ran out) in *status.
__global__ void k_selftest_wait(long long limit, int complete, uint32_t *status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t lane = threadIdx.x & 31;
    if (lane == 0) {
        mbar_init(&bar, 2);
        fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0 || (lane == 1 && complete)) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
    }
    __syncwarp();
    if (lane == 0) *status = mbar_wait_for(&bar, 0, limit) ? 1u : 2u;
}

}  // namespace

extern "C" rb_status rb_selftest_wait(uint64_t limit_cycles, int complete, void *stream) {
    clear_stale_error();
    if (limit_cycles == 0 || limit_cycles > (1ull << 31))
        return set_err(RB_EINVAL, "rb_selftest_wait: limit_cycles must be in [1, 2^31]");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *d = (uint32_t *)dev_alloc(sizeof(uint32_t), s);
    if (!d) return RB_ENOMEM;
    uint32_t h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, s>>>((long long)limit_cycles, complete ? 1 : 0, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(d, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_err(e, "rb_selftest_wait");
    if (h == 2u) return set_err(RB_ETIMEOUT, "rb_selftest_wait: the barrier wait ran out of its cycle limit");
    if (h != 1u) return set_err(RB_ECUDA, "rb_selftest_wait: the kernel left no status");
    return RB_OK;
}
