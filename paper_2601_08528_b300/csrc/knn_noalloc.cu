// knn_noalloc.cu -- svf_knn_static: the exact brute-force kNN of svf_knn for
// callers that cannot allocate device memory.
//
// Some callers of this library must not call cudaMalloc: a plugin or custom
// call inside a host framework whose memory manager owns all of the device's
// memory, or a latency-critical serving loop where an allocation could stall
// or fail.  svf_knn needs a caller-allocated key buffer of nq*k uint64; this
// variant keeps that scratch in a fixed device array instead.
//
// The array is a file-scope __device__ variable of kStaticKnnKeys keys (8 MiB);
// every GPU that loads the library holds it until the process exits.  Host
// code cannot use the array's name as a device address (on the host it names
// a host-side shadow), so the device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, and cached.  The
// cached address belongs to the device's primary context: after that context
// is torn down (cudaDeviceReset) it is stale, like every other device pointer
// the caller held.
#include <cstdio>
#include <mutex>

#include "index_impl.h"
#include "svf_internal.h"

namespace {

constexpr int64_t kStaticKnnKeys = 1 << 20;
static __device__ __align__(256) uint64_t g_knn_scratch[kStaticKnnKeys];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t *g_addr[kMaxDevices] = {};

thread_local char g_msg[256];

// The message goes to svf_knn_static_error() and, like every other entry
// point's, to svf_last_error().
int fail_static(int code, const char *msg) {
    snprintf(g_msg, sizeof g_msg, "svf_knn_static: %s", msg);
    return svf::fail(code, "%s", g_msg);
}

// Device address of the scratch array on the current device (set-up on the
// first call per device; later calls only read the cache).
int scratch_on_current_device(uint64_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_static(SVF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail_static(SVF_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_knn_scratch);
        if (e != cudaSuccess) return fail_static(SVF_ECUDA, cudaGetErrorString(e));
        g_addr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_addr[dev];
    return SVF_OK;
}

}  // namespace

extern "C" {

int64_t svf_knn_static_capacity(void) { return kStaticKnnKeys; }

const char *svf_knn_static_error(void) { return g_msg; }

int svf_knn_static(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t metric, const void *Q, int64_t nq,
                   const int64_t *self, int32_t k, uint32_t *out_ids, void *out_dist, void *stream) {
    if (n < 1 || nq < 0 || d < 16 || d > 2048 || d % 16 || k < 1 || k > 128)
        return fail_static(SVF_EINVAL, "bad sizes (n >= 1, d multiple of 16 in 16..2048, 1 <= k <= 128)");
    if (dtype != SVF_F32 && dtype != SVF_U8) return fail_static(SVF_EINVAL, "dtype must be F32 or U8");
    if (metric != SVF_L2 && metric != SVF_IP) return fail_static(SVF_EINVAL, "bad metric");
    if (nq > kStaticKnnKeys / k)
        return fail_static(SVF_EINVAL, "nq * k exceeds the static scratch of 1048576 keys; use svf_knn");
    if (nq == 0) return SVF_OK;
    if (!X || !Q || !out_ids) return fail_static(SVF_EINVAL, "null pointers");
    uint64_t *keys = nullptr;
    int rc = scratch_on_current_device(&keys);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    svf::KnnArgs a{};
    a.X.base = reinterpret_cast<const uint8_t *>(X);
    a.X.pitch = (int64_t)d * (dtype == SVF_U8 ? 1 : 4);
    a.X.nchunk = (int)(a.X.pitch / 16);
    a.X.d = d;
    a.X.dtype = dtype;
    a.X.metric = metric;
    a.X.copy_bytes = (int)a.X.pitch;
    a.n = n;
    a.Q = Q;
    a.q_row_bytes = (int)a.X.pitch;
    a.nq = nq;
    a.self = self;
    a.self_base = -1;
    a.k = k;
    a.out_keys = keys;  // every one of the nq*k keys is written: nothing to clear first
    cudaError_t e = svf::launch_knn(a, st);
    if (e == cudaSuccess)
        e = svf::launch_keys_to_out(keys, nq, k, k, dtype, metric, out_ids, reinterpret_cast<uint32_t *>(out_dist), st);
    if (e != cudaSuccess) return fail_static(SVF_ECUDA, cudaGetErrorString(e));
    return SVF_OK;
}

}  // extern "C"
