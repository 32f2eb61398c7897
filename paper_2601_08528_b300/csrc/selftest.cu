// selftest.cu -- the library's self-measurements.
//  * The failure path every device wait in the library shares: a bounded
//    poll of an mbarrier that gives up, records SVF_ETIMEOUT in the caller's
//    status words and returns, leaving the context usable.  Nothing arrives
//    at the barrier here, so the wait always runs out.
//  * The random-row fetch ceiling: the search kernel's row-copy pattern (one
//    bulk copy per lane, 32 rows per warp batch on one mbarrier) over random
//    ids, with no arithmetic, timed on the device.
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

constexpr int kProbeWarps = 4;   // warps per block
constexpr int kProbeBatch = 32;  // rows per warp batch (one per lane)

// Each warp: `iters` batches of 32 rows at random ids, one bulk copy per
// lane, completion counted in bytes on the warp's mbarrier.  A wait that gives
// up records SVF_ETIMEOUT, waits (bounded again) for the warp's own copies and
// returns.
__global__ void gather_probe_kernel(const uint8_t *__restrict__ tab, uint32_t n, int pitch, int cb, int iters,
                                    uint64_t seed, unsigned long long *status) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint8_t *buf = smem + (size_t)w * kProbeBatch * cb;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)kProbeWarps * kProbeBatch * cb) + w;
    if (lane == 0) mbar_init(bar, 1);
    __syncwarp();
    const uint64_t wkey = splitmix64(seed ^ splitmix64((uint64_t)blockIdx.x * kProbeWarps + w));
    uint32_t phase = 0;
    for (int it = 0; it < iters; it++) {
        __syncwarp();
        fence_proxy_async();
        if (lane == 0) mbar_expect_tx(bar, (uint32_t)(kProbeBatch * cb));
        __syncwarp();
        const uint32_t id = __umulhi((uint32_t)(splitmix64(wkey ^ ((uint64_t)it << 5 | (uint64_t)lane)) >> 32), n);
        bulk_g2s(buf + (size_t)lane * cb, tab + (int64_t)id * pitch, (uint32_t)cb, bar);
        uint32_t polls = 0;
        while (!mbar_try_wait(bar, phase)) {
            if (++polls > kWaitLimit) {
                if (lane == 0) set_error(status, SVF_ETIMEOUT, it);
                for (uint32_t k = 0; k < kWaitLimit && !mbar_try_wait(bar, phase); k++) {
                }
                return;
            }
        }
        phase ^= 1u;
    }
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

int svf_gather_probe(const void *table, int64_t n, int32_t pitch, int32_t row_bytes, int64_t rows, int32_t warps_per_sm,
                     uint64_t seed, unsigned long long *status, int64_t *out_rows, float *out_ms, void *stream) {
    if (!table || !status || !out_rows || !out_ms) return fail(SVF_EINVAL, "null table / status / outputs");
    if (reinterpret_cast<uintptr_t>(table) % 16) return fail(SVF_EINVAL, "table must be 16-byte aligned");
    if (pitch <= 0 || pitch % 16 || row_bytes < 16 || row_bytes % 16 || row_bytes > pitch || row_bytes > 1024)
        return fail(SVF_EINVAL, "need pitch, row_bytes multiples of 16 with 16 <= row_bytes <= min(pitch, 1024)");
    if (n < 1 || n >= ((int64_t)1 << 31)) return fail(SVF_EINVAL, "need 1 <= n < 2^31");
    if (rows < 1) return fail(SVF_EINVAL, "rows < 1");
    if (warps_per_sm < 4 || warps_per_sm > 64 || warps_per_sm % kProbeWarps)
        return fail(SVF_EINVAL, "warps_per_sm must be a multiple of 4 in [4, 64]");
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = sm_count() * warps_per_sm / kProbeWarps;
    const int64_t per_pass = (int64_t)blocks * kProbeWarps * kProbeBatch;
    const int64_t iters = (rows + per_pass - 1) / per_pass;
    if (iters > (1 << 26)) return fail(SVF_EINVAL, "rows too large for one launch");
    const size_t smem = (size_t)kProbeWarps * kProbeBatch * row_bytes + kProbeWarps * sizeof(uint64_t);
    CUDA_TRY(cudaFuncSetAttribute(gather_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(unsigned long long), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        gather_probe_kernel<<<blocks, kProbeWarps * 32, smem, st>>>(reinterpret_cast<const uint8_t *>(table),
                                                                   (uint32_t)n, pitch, row_bytes, (int)iters, seed, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, status, sizeof h, cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(SVF_ECUDA, "gather probe: %s", cudaGetErrorString(e));
    if (h) return fail(SVF_ETIMEOUT, "gather probe: a row-copy wait gave up");
    *out_rows = per_pass * iters;
    *out_ms = ms;
    return SVF_OK;
}

}  // extern "C"
