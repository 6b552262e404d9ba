// Self-test of the bounded waits of the tensor-core kernels (the paper has no
// counterpart).  One block initialises an mbarrier that nothing arrives on
// and waits on it with the same kind of %globaltimer deadline the MMA waits
// use; when the deadline passes it records a timeout and returns.  No tensor
// core, TMEM or memory outside the block is touched, so the context stays
// usable; the host reads the flag.
#include <cuda_runtime.h>

#include <cstdint>

#include "zeta_internal.h"

namespace zeta {

__global__ void k_wait_selftest(unsigned long long limit_ns, unsigned long long *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    unsigned long long waited = 0;
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(0u)
            : "memory");
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        waited = t - t0;
        if (done) { status[0] = 0; break; }
        if (waited > limit_ns) { status[0] = 1; break; }
    }
    status[1] = waited;
}

zeta_status wait_selftest(uint32_t limit_ms, double *waited_ms, std::string &err) {
    unsigned long long *d = nullptr, h[2] = {0, 0};
    cudaStream_t st = nullptr;  // legacy default stream of the current device
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) { cudaGetLastError(); err = "cudaMalloc"; return ZETA_ERR_OOM; }
    k_wait_selftest<<<1, 32, 0, st>>>((unsigned long long)limit_ms * 1000000ull, d);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(d);
    if (ce != cudaSuccess) { err = cudaGetErrorString(ce); return ZETA_ERR_DEVICE; }
    if (waited_ms) *waited_ms = (double)h[1] * 1e-6;
    if (h[0]) { err = "bounded wait gave up (expected)"; return ZETA_ERR_TIMEOUT; }
    return ZETA_OK;
}

}  // namespace zeta
