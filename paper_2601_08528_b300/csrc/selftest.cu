// selftest.cu -- exercises the failure path every device wait in the library
// shares: a bounded poll of an mbarrier that gives up, records SVF_ETIMEOUT
// in the caller's status words and returns, leaving the context usable.
// Nothing arrives at the barrier here, so the wait always runs out.
#include <chrono>

#include "index_impl.h"

namespace svf {
namespace {

__global__ void wait_timeout_kernel(uint32_t polls, unsigned long long *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t it = 0;
    bool done = true;
    while (!mbar_try_wait(&bar, 0))  // phase 0 never completes: no arrival is ever made
        if (++it > polls) {
            done = false;
            break;
        }
    if (!done && threadIdx.x == 0) set_error(status, SVF_ETIMEOUT, (long long)it);
}

}  // namespace
}  // namespace svf

using namespace svf;

extern "C" {

uint32_t svf_wait_limit(void) { return kWaitLimit; }

int svf_selftest_wait_timeout(uint32_t polls, unsigned long long *status, double *out_seconds, void *stream) {
    if (!status || polls == 0) return fail(SVF_EINVAL, "need a status buffer and polls >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(unsigned long long), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const auto t0 = std::chrono::steady_clock::now();
    wait_timeout_kernel<<<1, 32, 0, st>>>(polls, status);
    CUDA_TRY(cudaGetLastError());
    unsigned long long h[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(h, status, sizeof h, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (out_seconds) *out_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (h[0] == (unsigned long long)(unsigned)(-SVF_ETIMEOUT)) return SVF_ETIMEOUT;
    return fail(SVF_ECUDA, "the bounded wait did not report a timeout (status %llu)", h[0]);
}

}  // extern "C"
