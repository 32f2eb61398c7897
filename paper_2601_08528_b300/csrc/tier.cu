// tier.cu -- the tiered vector store of SVFusion's serving form (Sec. 4.2-4.4):
// all rows in pinned host memory, a device cache of M hot rows, the mapping
// table h_id -> cache slot, and workload-aware vector placement (WAVP,
// Alg. 2): miss counting with a sliding-window decay, Eq. 2's predicted
// access count F_lambda = alpha F_recent + beta log(1 + E_in), threshold
// promotion, and a clock sweep that evicts the unreferenced slot with the
// lowest F_lambda.  Maintenance runs between kernels (no search in flight),
// so a kernel never sees a slot change under it.
#include <algorithm>
#include <cmath>
#include <vector>

#include "index_impl.h"

namespace svf {
namespace {

constexpr int kHistBins = 4096;
constexpr uint32_t kMaxQueue = 16384, kMaxSweep = 8192;

__device__ __forceinline__ float flambda(float alpha, float beta, uint32_t freq, uint32_t ein) {
    return alpha * (float)(freq & ~kQueuedBit) + beta * log1pf((float)ein);
}

__global__ void ein_kernel(const uint32_t *graph, int64_t n_used, int R, const uint32_t *del, uint32_t *ein) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_used * R) return;
    const uint32_t t = graph[i];
    if (t == kEmpty || (int64_t)t >= n_used || is_deleted(del, t)) return;
    atomicAdd(ein + t, 1u);
}

__global__ void hist_kernel(const uint32_t *ein, int64_t n, unsigned long long *hist) {
    __shared__ unsigned int h[kHistBins];
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[min(ein[u], (uint32_t)kHistBins - 1)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Cold start: cache every id with E_in above the threshold bin and `quota`
// ids of the threshold bin.
__global__ void warm_assign_kernel(const uint32_t *ein, int64_t n, uint32_t thr, unsigned long long quota,
                                   int32_t *map, int32_t *owner, unsigned long long *cnt) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const uint32_t e = min(ein[u], (uint32_t)kHistBins - 1);
    bool take = e > thr;
    if (!take && e == thr) take = atomicAdd(cnt + 1, 1ull) < quota;
    if (!take) return;
    const unsigned long long s = atomicAdd(cnt, 1ull);
    map[u] = (int32_t)s;
    owner[s] = (int32_t)u;
}

// Warp per slot: copy row owner[s] from `src` rows into cache slot s.
__global__ void fill_slots_kernel(const uint8_t *src, int64_t pitch, const int32_t *owner, int64_t nslots,
                                  uint8_t *cache) {
    const int lane = threadIdx.x & 31;
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nslots) return;
    const int32_t o = owner[s];
    if (o < 0) return;
    const uint4 *a = reinterpret_cast<const uint4 *>(src + (int64_t)o * pitch);
    uint4 *b = reinterpret_cast<uint4 *>(cache + s * pitch);
    for (int c = lane; c < pitch / 16; c += 32) b[c] = a[c];
}

// Promotion candidates ordered by descending F_lambda (ties by id).
// by_order (CLOCK): in queue (miss) order instead.
__global__ void score_queue_kernel(const uint32_t *queue, int64_t c, int64_t npow, const uint32_t *freq,
                                   const uint32_t *ein, float alpha, float beta, int by_order, uint64_t *keys,
                                   float *fsum) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow) return;
    if (i >= c) {
        keys[i] = kPad;
        return;
    }
    const uint32_t x = queue[i];
    const float f = flambda(alpha, beta, freq[x], ein[x]);
    keys[i] = by_order ? make_key((uint32_t)i, x) : make_key(~fkey(f), x);
    atomicAdd(fsum, f);
}

// Clock sweep over W slots from the hand: referenced slots lose their bit;
// unreferenced ones become victims ordered by ascending F_lambda of their
// owner (empty slots first), or (by_order: CLOCK) in the order the clock
// meets them.
__global__ void victim_kernel(const int32_t *owner, uint8_t *ref, const uint32_t *freq, const uint32_t *ein,
                              int64_t M, int64_t hand, int64_t W, int64_t npow, float alpha, float beta,
                              int by_order, uint64_t *keys, unsigned long long *nvalid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow) return;
    if (i >= W) {
        keys[i] = kPad;
        return;
    }
    const int64_t s = (hand + i) % M;
    if (ref[s]) {
        ref[s] = 0;
        keys[i] = kPad;
        return;
    }
    const int32_t o = owner[s];
    if (by_order) {
        keys[i] = make_key(o < 0 ? 0u : (uint32_t)i + 1u, (uint32_t)s);
    } else {
        const float f = o < 0 ? -INFINITY : flambda(alpha, beta, freq[o], ein[o]);
        keys[i] = make_key(fkey(f), (uint32_t)s);
    }
    atomicAdd(nvalid, 1ull);
}

// LRU / LRFU victims: every slot of the window, ordered by the last-hit stamp
// (LRU) or by C (LRFU), ascending; an empty slot first; ties by slot.
__global__ void victim_recency_kernel(const int32_t *owner, const uint32_t *stat, int lru, int64_t M, int64_t hand,
                                      int64_t W, int64_t npow, uint64_t *keys, unsigned long long *nvalid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npow) return;
    if (i >= W) {
        keys[i] = kPad;
        return;
    }
    const int64_t s = (hand + i) % M;
    uint32_t k;
    if (owner[s] < 0)
        k = 0u;
    else if (lru)
        k = stat[2 * s] + 1u;  // stamps are below 2^32 - 1
    else
        k = fkey(__uint_as_float(stat[2 * s + 1]));  // C >= 0 sorts after the empty key 0
    keys[i] = make_key(k, (uint32_t)s);
    atomicAdd(nvalid, 1ull);
}

// LRFU: fold the round's hits into C (C <- C * 2^-lambda + hits) for every slot.
__global__ void lrfu_fold_kernel(uint32_t *stat, int64_t M, float decay) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const float c = __uint_as_float(stat[2 * s + 1]) * decay + (float)stat[2 * s];
    stat[2 * s + 1] = __float_as_uint(c);
    stat[2 * s] = 0u;
}

// Recency state of the slots just filled: LRU stamp = this round's tick,
// LRFU C = 1 (the miss that admitted the row).
__global__ void promoted_stat_kernel(const uint64_t *promo, const uint64_t *victims, int64_t nb, uint32_t *stat,
                                     int lru, uint32_t tick) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const uint64_t pk = promo[i], vk = victims[i];
    if (key_is_pad(pk) || key_is_pad(vk)) return;
    const uint32_t s = (uint32_t)vk;
    if (lru) {
        stat[2 * (int64_t)s] = tick;
    } else {
        stat[2 * (int64_t)s] = 0u;
        stat[2 * (int64_t)s + 1] = __float_as_uint(1.f);
    }
}

// Single-CTA ascending bitonic sort of npow (power of two, <= 16384) keys.
__global__ void __launch_bounds__(1024) sort_kernel(uint64_t *keys, int npow) {
    extern __shared__ uint64_t sk[];
    for (int i = threadIdx.x; i < npow; i += blockDim.x) sk[i] = keys[i];
    __syncthreads();
    for (int size = 2; size <= npow; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < npow; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool asc = (i & size) == 0;
                    const uint64_t a = sk[i], b = sk[j];
                    if ((a > b) == asc) {
                        sk[i] = b;
                        sk[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < npow; i += blockDim.x) keys[i] = sk[i];
}

// Warp per (candidate i, victim i): remap and copy the host row into the slot.
__global__ void apply_kernel(const uint64_t *promo, const uint64_t *victims, int64_t nb, int32_t *map, int32_t *owner,
                             uint8_t *ref, const uint8_t *host, uint8_t *cache, int64_t pitch,
                             unsigned long long *status) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= nb) return;
    const uint64_t pk = promo[i], vk = victims[i];
    if (key_is_pad(pk) || key_is_pad(vk)) return;
    const uint32_t x = (uint32_t)pk, s = (uint32_t)vk;
    if (lane == 0) {
        const int32_t old = owner[s];
        if (old >= 0) {
            map[old] = -1;
            atomicAdd(status + kStEvicted, 1ull);
        }
        owner[s] = (int32_t)x;
        map[x] = (int32_t)s;
        ref[s] = 1;
        atomicAdd(status + kStPromoted, 1ull);
    }
    const uint4 *a = reinterpret_cast<const uint4 *>(host + (int64_t)x * pitch);
    uint4 *b = reinterpret_cast<uint4 *>(cache + (int64_t)s * pitch);
    for (int c = lane; c < pitch / 16; c += 32) b[c] = a[c];
}

__global__ void unqueue_kernel(const uint32_t *queue, int64_t c, uint32_t *freq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < c) atomicAnd(freq + queue[i], ~kQueuedBit);
}

__global__ void decay_kernel(uint32_t *freq, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint32_t f = freq[i];
        freq[i] = (f & kQueuedBit) | ((f & ~kQueuedBit) >> 1);
    }
}

int64_t pow2_at_least(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// Parameters, cleared tables, E_in from the graph, and the cold-start cache
// of the highest in-degree rows (rows read from `src`: the device store at
// enable, the host store at reset).  Synchronises the stream.
int tier_init(svf_index *h, const svf_tier_params *tp, const uint8_t *src, cudaStream_t st) {
    Tier &T = h->tier;
    const int64_t n = h->n_used, R = h->p.R;
    const int64_t pitch = (int64_t)h->p.d * esize_of(h->p.dtype);
    T.qcap = tp->qcap;
    T.alpha = tp->alpha;
    T.beta = tp->beta;
    T.theta = T.theta0 = tp->theta0;
    T.promote_batch = tp->promote_batch;
    T.sweep = tp->sweep;
    T.decay_every = tp->decay_every ? tp->decay_every : (1ull << 16);
    T.policy = tp->policy;
    T.M = tp->M;
    T.lambda = tp->lrfu_lambda > 0.f ? tp->lrfu_lambda : 0.5f;
    T.tick = 0;
    T.clock = 0;
    T.rounds = 0;
    T.last_rate = T.last_meanf = 0.0;
    CUDA_TRY(cudaMemsetAsync(T.map, 0xFF, (size_t)h->p.n_cap * 4, st));
    CUDA_TRY(cudaMemsetAsync(T.owner, 0xFF, (size_t)T.M * 4, st));
    CUDA_TRY(cudaMemsetAsync(T.ref, 0, (size_t)T.M, st));
    CUDA_TRY(cudaMemsetAsync(T.stat, 0, (size_t)T.M * 8, st));
    CUDA_TRY(cudaMemsetAsync(T.freq, 0, (size_t)h->p.n_cap * 4, st));
    CUDA_TRY(cudaMemsetAsync(T.ein, 0, (size_t)h->p.n_cap * 4, st));
    CUDA_TRY(cudaMemsetAsync(h->status() + kStQCount, 0, 8, st));
    if (n) {
        ein_kernel<<<grid_for(n * R, 256), 256, 0, st>>>(h->b.graph, n, (int)R, h->b.del_bits, T.ein);
        unsigned long long *hist = reinterpret_cast<unsigned long long *>(T.scratch + kMaxQueue + kMaxSweep);
        CUDA_TRY(cudaMemsetAsync(hist, 0, kHistBins * 8 + 16, st));
        hist_kernel<<<296, 256, 0, st>>>(T.ein, n, hist);
        std::vector<unsigned long long> hh(kHistBins);
        CUDA_TRY(cudaMemcpyAsync(hh.data(), hist, kHistBins * 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        unsigned long long above = 0;
        int thr = kHistBins - 1;
        const unsigned long long M = (unsigned long long)std::min<int64_t>(T.M, n);
        for (; thr >= 0; thr--) {
            if (above + hh[thr] >= M) break;
            above += hh[thr];
        }
        if (thr < 0) thr = 0;
        const unsigned long long quota = M - std::min(M, above);
        unsigned long long *cnt = hist + kHistBins;
        warm_assign_kernel<<<grid_for(n, 256), 256, 0, st>>>(T.ein, n, (uint32_t)thr, quota, T.map, T.owner, cnt);
        fill_slots_kernel<<<grid_for(T.M * 32, 256), 256, 0, st>>>(src, pitch, T.owner, T.M, T.cache);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(st));
    unsigned long long s[kStWords];
    CUDA_TRY(cudaMemcpy(s, h->status(), sizeof s, cudaMemcpyDeviceToHost));
    T.last_hits = s[kStHits];
    T.last_misses = T.misses_at_decay = s[kStMisses];
    return SVF_OK;
}

}  // namespace
}  // namespace svf

using namespace svf;

extern "C" {

int svf_tier_buffer_sizes(const svf_params *p, const svf_tier_params *tp, svf_tier_sizes *out) {
    if (!p || !tp || !out) return fail(SVF_EINVAL, "null arguments");
    if (tp->M < 1 || tp->M > p->n_cap) return fail(SVF_EINVAL, "cache slots M must be in [1, n_cap]");
    if (tp->qcap < 1 || tp->qcap > kMaxQueue) return fail(SVF_EINVAL, "qcap must be in [1, 16384]");
    if (tp->promote_batch < 1 || tp->promote_batch > 2048) return fail(SVF_EINVAL, "promote_batch in [1, 2048]");
    if (tp->sweep < 1 || (int64_t)tp->sweep * tp->promote_batch > kMaxSweep)
        return fail(SVF_EINVAL, "sweep * promote_batch must be <= 8192");
    if (tp->policy < SVF_TIER_WAVP || tp->policy > SVF_TIER_LRFU) return fail(SVF_EINVAL, "unknown tier policy");
    if (!(tp->lrfu_lambda >= 0.f)) return fail(SVF_EINVAL, "lrfu_lambda must be >= 0");
    const int64_t pitch = (int64_t)p->d * esize_of(p->dtype);
    out->cache = align256((size_t)tp->M * pitch);
    out->map = align256((size_t)p->n_cap * 4);
    out->owner = align256((size_t)tp->M * 4);
    out->ref = align256((size_t)tp->M);
    out->freq = align256((size_t)p->n_cap * 4);
    out->ein = align256((size_t)p->n_cap * 4);
    out->queue = align256((size_t)tp->qcap * 4);
    out->scratch = align256((size_t)(kMaxQueue + kMaxSweep) * 8 + kHistBins * 8 + 64);
    out->host = (size_t)p->n_cap * pitch;
    out->slot_stat = align256((size_t)tp->M * 8);
    return SVF_OK;
}

int svf_tier_enable(svf_index *h, const svf_tier_params *tp, const svf_tier_buffers *tb, void *stream) {
    if (!h || !tp || !tb) return fail(SVF_EINVAL, "null arguments");
    if (h->tier.on) return fail(SVF_EINVAL, "the store is already tiered");
    svf_tier_sizes sz;
    int rc = svf_tier_buffer_sizes(&h->p, tp, &sz);
    if (rc) return rc;
    if (!tb->cache || !tb->map || !tb->owner || !tb->ref || !tb->freq || !tb->ein || !tb->queue || !tb->scratch ||
        !tb->host || !tb->slot_stat)
        return fail(SVF_EINVAL, "a tier buffer is null");
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    Tier &T = h->tier;
    const int64_t n = h->n_used;
    const int64_t pitch = (int64_t)h->p.d * esize_of(h->p.dtype);
    T.host = reinterpret_cast<uint8_t *>(tb->host);
    T.cache = reinterpret_cast<uint8_t *>(tb->cache);
    T.M = tp->M;
    T.map = tb->map;
    T.owner = tb->owner;
    T.ref = tb->ref;
    T.freq = tb->freq;
    T.ein = tb->ein;
    T.queue = tb->queue;
    T.scratch = reinterpret_cast<uint64_t *>(tb->scratch);
    T.stat = reinterpret_cast<uint32_t *>(tb->slot_stat);
    T.M_alloc = tp->M;
    // host copy of the rows, then the tables and the warm cache
    if (n) CUDA_TRY(cudaMemcpyAsync(T.host, h->b.vecs, (size_t)n * pitch, cudaMemcpyDeviceToHost, st));
    rc = tier_init(h, tp, reinterpret_cast<const uint8_t *>(h->b.vecs), st);
    if (rc) return rc;
    T.on = true;
    return SVF_OK;
}

int svf_tier_reset(svf_index *h, const svf_tier_params *tp, void *stream) {
    if (!h || !tp) return fail(SVF_EINVAL, "null arguments");
    if (!h->tier.on) return fail(SVF_EINVAL, "the store is not tiered");
    if (tp->M > h->tier.M_alloc) return fail(SVF_EINVAL, "reset: M exceeds the slots the buffers hold");
    svf_tier_sizes sz;
    const int rc = svf_tier_buffer_sizes(&h->p, tp, &sz);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    return tier_init(h, tp, h->tier.host, st);
}

int svf_tier_maintain(svf_index *h, int64_t *out_promoted, void *stream) {
    if (!h) return fail(SVF_EINVAL, "null index");
    if (!h->tier.on) return fail(SVF_EINVAL, "the store is not tiered");
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    Tier &T = h->tier;
    unsigned long long s[kStWords];
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaMemcpy(s, h->status(), sizeof s, cudaMemcpyDeviceToHost));
    // STATIC keeps its cold-start cache (nothing is ever queued)
    const int64_t c = T.policy == SVF_TIER_STATIC ? 0 : (int64_t)std::min<unsigned long long>(s[kStQCount], T.qcap);
    const bool lr = T.policy == SVF_TIER_LRU || T.policy == SVF_TIER_LRFU;
    const int by_order = T.policy == SVF_TIER_CLOCK || lr;
    if (T.policy == SVF_TIER_LRFU && T.M > 0) {
        lrfu_fold_kernel<<<grid_for(T.M, 256), 256, 0, st>>>(T.stat, T.M, exp2f(-T.lambda));
        CUDA_TRY(cudaGetLastError());
    }
    const float wa = T.policy == SVF_TIER_WAVP ? T.alpha : 1.f, wb = T.policy == SVF_TIER_WAVP ? T.beta : 0.f;
    const unsigned long long prom0 = s[kStPromoted];
    float meanf = 0.f;
    const int64_t pitch = (int64_t)h->p.d * esize_of(h->p.dtype);
    if (c > 0) {
        uint64_t *pk = T.scratch;
        uint64_t *vk = T.scratch + kMaxQueue;
        float *fsum = reinterpret_cast<float *>(T.scratch + kMaxQueue + kMaxSweep + kHistBins + 2);
        const int64_t np = pow2_at_least(c);
        const int64_t B = std::min<int64_t>(c, T.promote_batch);
        const int64_t W = std::min<int64_t>((int64_t)T.sweep * B, T.M);
        const int64_t nw = pow2_at_least(W);
        CUDA_TRY(cudaMemsetAsync(fsum, 0, 4, st));
        score_queue_kernel<<<grid_for(np, 256), 256, 0, st>>>(T.queue, c, np, T.freq, T.ein, wa, wb, by_order, pk,
                                                               fsum);
        cudaFuncSetAttribute(sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxQueue * 8));
        sort_kernel<<<1, 1024, np * 8, st>>>(pk, (int)np);
        // the clock passes over the window; if too few slots were unreferenced
        // it comes round again (all reference bits are clear by then)
        unsigned long long *nvalid = reinterpret_cast<unsigned long long *>(fsum + 2);
        CUDA_TRY(cudaMemsetAsync(nvalid, 0, 8, st));
        if (lr) {
            victim_recency_kernel<<<grid_for(nw, 256), 256, 0, st>>>(T.owner, T.stat, T.policy == SVF_TIER_LRU, T.M,
                                                                      T.clock, W, nw, vk, nvalid);
        } else {
            victim_kernel<<<grid_for(nw, 256), 256, 0, st>>>(T.owner, T.ref, T.freq, T.ein, T.M, T.clock, W, nw, wa,
                                                              wb, by_order, vk, nvalid);
            unsigned long long nv = 0;
            CUDA_TRY(cudaMemcpyAsync(&nv, nvalid, 8, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if ((int64_t)nv < B)
                victim_kernel<<<grid_for(nw, 256), 256, 0, st>>>(T.owner, T.ref, T.freq, T.ein, T.M, T.clock, W, nw,
                                                                  wa, wb, by_order, vk, nvalid);
        }
        sort_kernel<<<1, 1024, nw * 8, st>>>(vk, (int)nw);
        apply_kernel<<<grid_for(B * 32, 256), 256, 0, st>>>(pk, vk, B, T.map, T.owner, T.ref, T.host, T.cache, pitch,
                                                             h->status());
        if (lr)
            promoted_stat_kernel<<<grid_for(B, 256), 256, 0, st>>>(pk, vk, B, T.stat, T.policy == SVF_TIER_LRU,
                                                                    T.tick);
        unqueue_kernel<<<grid_for(c, 256), 256, 0, st>>>(T.queue, c, T.freq);
        CUDA_TRY(cudaMemsetAsync(h->status() + kStQCount, 0, 8, st));
        CUDA_TRY(cudaGetLastError());
        T.clock = (T.clock + W) % T.M;
        CUDA_TRY(cudaMemcpyAsync(&meanf, fsum, 4, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        meanf /= (float)c;
    }
    // sliding window: halve F_recent every decay_every misses
    if (s[kStMisses] - T.misses_at_decay >= T.decay_every) {
        decay_kernel<<<grid_for(h->n_used, 256), 256, 0, st>>>(T.freq, h->n_used);
        CUDA_TRY(cudaGetLastError());
        T.misses_at_decay = s[kStMisses];
    }
    // adaptive threshold (Sec. 4.4): more selective when the miss rate and the
    // predicted access counts of the candidates both rose
    const double acc = (double)(s[kStHits] - T.last_hits) + (double)(s[kStMisses] - T.last_misses);
    const double rate = acc > 0 ? (double)(s[kStMisses] - T.last_misses) / acc : 0.0;
    if (T.rounds > 0 && T.policy == SVF_TIER_WAVP) {
        if (rate > T.last_rate && meanf > T.last_meanf)
            T.theta *= 1.25f;
        else
            T.theta *= 0.95f;
        T.theta = std::min(std::max(T.theta, T.theta0 / 8.f), T.theta0 * 8.f);
    }
    T.last_rate = rate;
    T.last_meanf = meanf;
    T.last_hits = s[kStHits];
    T.last_misses = s[kStMisses];
    T.rounds++;
    if (out_promoted) {
        unsigned long long p1 = 0;
        CUDA_TRY(cudaMemcpyAsync(&p1, h->status() + kStPromoted, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        *out_promoted = (int64_t)(p1 - prom0);
    }
    return SVF_OK;
}

float svf_tier_theta(svf_index *h) { return h && h->tier.on ? h->tier.theta : 0.f; }

}  // extern "C"
