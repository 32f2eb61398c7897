// knn.cu -- exact brute-force k nearest neighbours by (distance, id): the
// 2R-NN lists of the build (Sec. 3 "Build", Sec. 4.2) and ground truth by
// exhaustive scan (Sec. 6.1).  SIMT: fp32 FMA, or exact int32 for uint8
// (|a-b| per byte with __vabsdiffu4, squares summed by __dp4a).
//
// A CTA owns 32 queries and streams the database (or one slice of it) in tiles of 64 rows; each
// thread accumulates a 2 x 4 block of distances from transposed shared-memory
// tiles (32 words of the row per step).  Candidates below a query's current
// k-th key are appended to a per-query buffer; after each tile one warp per
// query sorts the buffer and merges it into the query's 128-entry list.
#include <algorithm>
#include <cstdint>

#include "svf_internal.h"

namespace svf {

namespace {
constexpr int QB = 32, NB = 64, WC = 32;  // queries, rows, 32-bit words per step
constexpr int KMAX = 128;
constexpr int THREADS = 256;

// Rows [blockIdx.y * slice, ...) of the store when slice > 0 (out: [nq][gridDim.y][k]), else all rows
// (out: [nq][k]).
template <int DT>
__global__ void __launch_bounds__(THREADS) knn_kernel(const KnnArgs a, int64_t slice, uint64_t *out) {
    extern __shared__ __align__(16) uint8_t sm[];
    uint64_t(*lists)[KMAX] = reinterpret_cast<uint64_t(*)[KMAX]>(sm);
    uint64_t(*buf)[NB] = reinterpret_cast<uint64_t(*)[NB]>(sm + sizeof(uint64_t) * QB * KMAX);
    uint64_t *thr = reinterpret_cast<uint64_t *>(sm + sizeof(uint64_t) * QB * (KMAX + NB));
    uint32_t(*Qs)[QB + 1] = reinterpret_cast<uint32_t(*)[QB + 1]>(sm + sizeof(uint64_t) * QB * (KMAX + NB + 1));
    uint32_t(*Xs)[NB + 1] = reinterpret_cast<uint32_t(*)[NB + 1]>(reinterpret_cast<uint8_t *>(Qs) +
                                                                   sizeof(uint32_t) * WC * (QB + 1));
    int *cnt = reinterpret_cast<int *>(reinterpret_cast<uint8_t *>(Xs) + sizeof(uint32_t) * WC * (NB + 1));

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tq = tid >> 4, tn = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * QB;
    const int words = a.q_row_bytes / 4;  // 32-bit words of a row's values

    for (int i = tid; i < QB * KMAX; i += THREADS) lists[i / KMAX][i % KMAX] = kPad;
    if (tid < QB) {
        cnt[tid] = 0;
        thr[tid] = kPad;
    }
    int64_t selfq[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        int64_t q = q0 + tq + 16 * i;
        selfq[i] = q >= a.nq ? -1 : a.self ? a.self[q] : a.self_base >= 0 ? a.self_base + q : -1;
    }
    __syncthreads();

    const int64_t r_begin = slice > 0 ? (int64_t)blockIdx.y * slice : 0;
    const int64_t r_end = slice > 0 ? (r_begin + slice < a.n ? r_begin + slice : a.n) : a.n;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += NB) {
        float facc[2][4];
        uint32_t iacc[2][4];
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                facc[i][j] = 0.f;
                iacc[i][j] = 0u;
            }
        for (int w0 = 0; w0 < words; w0 += WC) {
            for (int i = tid; i < QB * WC; i += THREADS) {
                int q = i / WC, w = i % WC;
                int64_t gq = q0 + q;
                Qs[w][q] = (gq < a.nq && w0 + w < words)
                               ? __ldg(reinterpret_cast<const uint32_t *>(a.Q) + gq * words + w0 + w)
                               : 0u;
            }
            for (int i = tid; i < NB * WC; i += THREADS) {
                int r = i / WC, w = i % WC;
                int64_t gr = r0 + r;
                Xs[w][r] = (gr < r_end && w0 + w < words)
                               ? __ldg(reinterpret_cast<const uint32_t *>(a.X.base + gr * a.X.pitch) + w0 + w)
                               : 0u;
            }
            __syncthreads();
#pragma unroll 8
            for (int w = 0; w < WC; w++) {
                uint32_t qv[2] = {Qs[w][tq], Qs[w][tq + 16]};
                uint32_t xv[4] = {Xs[w][tn], Xs[w][tn + 16], Xs[w][tn + 32], Xs[w][tn + 48]};
#pragma unroll
                for (int i = 0; i < 2; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if constexpr (DT == SVF_U8) {
                            if (a.X.metric == SVF_L2) {
                                uint32_t df = __vabsdiffu4(qv[i], xv[j]);
                                iacc[i][j] = __dp4a(df, df, iacc[i][j]);
                            } else {
                                iacc[i][j] = __dp4a(qv[i], xv[j], iacc[i][j]);
                            }
                        } else {
                            float qf = __uint_as_float(qv[i]), xf = __uint_as_float(xv[j]);
                            if (a.X.metric == SVF_L2) {
                                float df = qf - xf;
                                facc[i][j] = fmaf(df, df, facc[i][j]);
                            } else {
                                facc[i][j] = fmaf(qf, xf, facc[i][j]);
                            }
                        }
                    }
            }
            __syncthreads();
        }
        // filter into the per-query buffers
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int ql = tq + 16 * i;
            if (q0 + ql >= a.nq) continue;
            const uint64_t th = thr[ql];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                int64_t gr = r0 + tn + 16 * j;
                if (gr >= r_end || gr == selfq[i]) continue;
                if (a.del && is_deleted(a.del, (uint32_t)gr)) continue;
                uint32_t dk;
                if constexpr (DT == SVF_U8)
                    dk = a.X.metric == SVF_L2 ? iacc[i][j] : ((uint32_t)(-(int32_t)iacc[i][j]) ^ 0x80000000u);
                else
                    dk = fkey(a.X.metric == SVF_L2 ? facc[i][j] : -facc[i][j]);
                uint64_t key = make_key(dk, (uint32_t)gr);
                if (cmpk(key) < cmpk(th)) {
                    int p = atomicAdd(&cnt[ql], 1);
                    buf[ql][p] = key;
                }
            }
        }
        __syncthreads();
        for (int ql = warp; ql < QB; ql += THREADS / 32) {
            const int c = cnt[ql];
            if (c == 0) continue;
            uint64_t cand[2] = {lane < c ? buf[ql][lane] : kPad, lane + 32 < c ? buf[ql][lane + 32] : kPad};
            warp_sort<2>(cand, lane);
            uint64_t lst[4];
#pragma unroll
            for (int s = 0; s < 4; s++) lst[s] = lists[ql][s * 32 + lane];
            warp_merge_into<4, 2>(lst, cand, lane);
#pragma unroll
            for (int s = 0; s < 4; s++) lists[ql][s * 32 + lane] = lst[s];
            __syncwarp();
            if (lane == 0) {
                thr[ql] = lists[ql][a.k - 1];
                cnt[ql] = 0;
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < QB * a.k; i += THREADS) {
        int ql = i / a.k, j = i % a.k;
        if (q0 + ql < a.nq) out[((q0 + ql) * gridDim.y + blockIdx.y) * a.k + j] = lists[ql][j];
    }
}

// Warp per query: the best k of its s sorted slice lists (s * k <= 512 keys).
__global__ void merge_slices_kernel(const uint64_t *part, int64_t nq, int s, int k, uint64_t *out) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    uint64_t v[16];
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const int e = t * 32 + lane;
        v[t] = e < s * k ? part[q * s * k + e] : kPad;
    }
    warp_sort<16>(v, lane);
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int e = t * 32 + lane;
        if (e < k) out[q * k + e] = v[t];
    }
}

__global__ void keys_to_out_kernel(const uint64_t *keys, int64_t nq, int kin, int kout, int dtype, int metric,
                                   uint32_t *ids, uint32_t *dist) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq * kout) return;
    int64_t q = i / kout;
    int j = (int)(i % kout);
    uint64_t k = keys[q * kin + j];
    bool pad = key_is_pad(k);
    ids[i] = pad ? kEmpty : key_id(k);
    if (dist) dist[i] = key_to_out(pad ? 0xFFFFFFFFu : (uint32_t)(k >> 32), dtype, metric);
}
}  // namespace

cudaError_t launch_knn(const KnnArgs &a, cudaStream_t st) {
    if (a.k < 1 || a.k > KMAX || a.nq <= 0) return cudaErrorInvalidValue;
    const int64_t qtiles = (a.nq + QB - 1) / QB;
    const size_t smem = sizeof(uint64_t) * QB * (KMAX + NB + 1) + sizeof(uint32_t) * WC * (QB + 1) +
                        sizeof(uint32_t) * WC * (NB + 1) + sizeof(int) * QB;
    // slices: enough blocks for about three per SM, each slice list k keys,
    // all of a query's slice lists together at most 512 keys, within the scratch
    int s = 1;
    if (a.part_keys) {
        const int64_t want = ((int64_t)3 * sm_count() + qtiles - 1) / qtiles;
        const int64_t fit = (int64_t)(a.part_bytes / ((size_t)a.nq * a.k * sizeof(uint64_t)));
        s = (int)std::min<int64_t>(std::min<int64_t>(want, 512 / a.k), std::min<int64_t>(fit, 16));
        if (s < 2) s = 1;
    }
    const int64_t slice = s > 1 ? ((a.n + s - 1) / s + NB - 1) / NB * NB : 0;
    dim3 grid((unsigned)qtiles, (unsigned)s);
    uint64_t *out = s > 1 ? a.part_keys : a.out_keys;
    if (a.X.dtype == SVF_U8) {
        cudaFuncSetAttribute(knn_kernel<SVF_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        knn_kernel<SVF_U8><<<grid, THREADS, smem, st>>>(a, slice, out);
    } else {
        cudaFuncSetAttribute(knn_kernel<SVF_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        knn_kernel<SVF_F32><<<grid, THREADS, smem, st>>>(a, slice, out);
    }
    if (s > 1) merge_slices_kernel<<<(unsigned)((a.nq * 32 + 255) / 256), 256, 0, st>>>(a.part_keys, a.nq, s, a.k,
                                                                                         a.out_keys);
    return cudaGetLastError();
}

cudaError_t launch_knn_self(const RowDesc &X, int64_t n, int64_t q0, int64_t nq, int k, uint64_t *out_keys,
                            cudaStream_t st) {
    // queries are rows of the store itself; the store pitch equals the row
    // bytes for the primary dtypes, so the store is also a dense query array
    KnnArgs a{};
    a.X = X;
    a.n = n;
    a.Q = X.base + q0 * X.pitch;
    a.q_row_bytes = (int)X.pitch;
    a.nq = nq;
    a.self = nullptr;
    a.self_base = q0;
    a.del = nullptr;
    a.k = k;
    a.out_keys = out_keys;
    return launch_knn(a, st);
}

cudaError_t launch_keys_to_out(const uint64_t *keys, int64_t nq, int kin, int kout, int dtype, int metric,
                               uint32_t *ids, uint32_t *dist, cudaStream_t st) {
    int64_t n = nq * kout;
    if (n == 0) return cudaSuccess;
    keys_to_out_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, nq, kin, kout, dtype, metric, ids, dist);
    return cudaGetLastError();
}

}  // namespace svf
