// Diagnostics: the bounded device wait that every pipelined kernel of the library relies on,
// exercised on its own so that its time-out path (status word -> YF_E_TIMEOUT on the host,
// context still usable) can be tested without faulting or hanging a GPU.
#include <cuda_runtime.h>

#include "yf_internal.h"

namespace yf {
namespace {

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// one thread waits for *flag != 0 for at most limit_ns; on expiry it records 1 in *status
__global__ void k_wait_flag(const volatile int *flag, unsigned long long limit_ns, int *status)
{
    const unsigned long long t0 = now_ns();
    while (*flag == 0) {
        if (now_ns() - t0 > limit_ns) {
            *status = 1;
            return;
        }
        __nanosleep(1000);
    }
    *status = 0;
}

}  // namespace
}  // namespace yf

extern "C" yf_status yf_bounded_wait_check(int preset_flag, double limit_seconds)
{
    using namespace yf;
    if (!(limit_seconds > 0) || limit_seconds > 10.0)
        return fail(YF_E_INVALID, "yf_bounded_wait_check: limit must be in (0, 10] s");
    int *buf = nullptr;
    YF_CUDA_TRY(cudaMalloc(&buf, 2 * sizeof(int)));
    const int init[2] = {preset_flag ? 1 : 0, -1};
    cudaError_t e = cudaMemcpy(buf, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_wait_flag<<<1, 1>>>(buf, (unsigned long long)(limit_seconds * 1e9), buf + 1);
        e = cudaGetLastError();
    }
    int out[2] = {0, -1};
    if (e == cudaSuccess) e = cudaMemcpy(out, buf, sizeof(out), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "yf_bounded_wait_check");
    if (out[1] == 1) return fail(YF_E_TIMEOUT, "device wait gave up after %.3f s (flag never set)", limit_seconds);
    if (out[1] != 0) return fail(YF_E_CUDA, "yf_bounded_wait_check: the wait kernel did not run");
    return YF_OK;
}
