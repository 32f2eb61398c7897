// tc_knn.cu -- exact brute-force k nearest neighbours on the tensor cores
// (ground truth, Sec. 6.1 "exhaustive linear scan"), for fp32 stores with
// d <= 128.
//
// 1. Rows and queries are rounded to bf16 (zero-padded to 128 columns).
// 2. tc_knn_kernel: a CTA owns 128 queries and one slice of the database.
//    TMA loads 128-byte-swizzled tiles (queries once, 256 database rows per
//    stage, two stages); one thread issues tcgen05.mma (kind::f16, bf16 in,
//    fp32 accumulate, M=128, N=256, K=16) into a double-buffered TMEM
//    accumulator; the four warps read their 32 TMEM lanes (= queries) with
//    tcgen05.ld and keep each query's 48 best approximate distances.  The
//    MMA of tile t+1 runs while tile t is scanned.
// 3. rescore_kernel: per query, the candidates of all slices get exact fp32
//    distances and the best k by (distance, id) are kept.  A certificate
//    checks the result: every row left out of a slice's candidates has an
//    approximate distance at least that slice's 48th, and the bf16 error of
//    a distance is at most c ||q|| ||x|| (c = 2^-7 + d 2^-24 for the
//    products and the fp32 sums, doubled for L2), so if min_slice(48th) - eps
//    exceeds the k-th exact distance no row can be missing.  Queries that
//    fail it are recomputed by the SIMT kernel (knn.cu).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>

#include "index_impl.h"

namespace svf {
namespace {

constexpr int TM = 128, TN = 128, KP = 128, KC = 48, THREADS = 128;
constexpr int NS = 4;                  // database tile stages in flight
constexpr int A_BYTES = TM * KP * 2;   // two 64-column swizzle atoms of 128 rows
constexpr int B_STAGE = TN * KP * 2;   // two atoms of TN rows
constexpr int LIST_BYTES = KC * TM * 8;
constexpr int NBAR = 1 + NS + 2;       // A, B stages, MMA done (two TMEM halves)
constexpr int SMEM_BYTES = 1024 + A_BYTES + NS * B_STAGE + LIST_BYTES + 8 * NBAR + 64;
constexpr uint32_t kTmemCols = 2 * TN;

struct TcArgs {
    int64_t n, nq;
    int64_t rows_per_split;
    int splits;
    int metric;
    const float *norms;  // ||x||^2 (L2)
    float *cand_d;       // [nq][splits][KC]
    uint32_t *cand_i;
    unsigned long long *status;
};

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: kind::f16, bf16 x bf16 -> fp32, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            tmem_d),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity) {
    uint32_t it = 0;
    while (!mbar_try_wait(bar, parity))
        if (++it > kWaitLimit) return false;
    return true;
}

#define TMEM_LD32(taddr, v)                                                                                           \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"  \
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                        \
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),    \
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),           \
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),         \
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),         \
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                                                                \
                 : "r"(taddr))

__global__ void __launch_bounds__(THREADS, 1)
    tc_knn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
    extern __shared__ uint8_t sm_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;
    uint8_t *sB = sm + A_BYTES;
    float *ld = reinterpret_cast<float *>(sB + NS * B_STAGE);
    uint32_t *li = reinterpret_cast<uint32_t *>(ld + KC * TM);
    uint64_t *bar = reinterpret_cast<uint64_t *>(li + KC * TM);  // 0: A, 1..NS: B stages, NS+1..NS+2: MMA done
    uint64_t *mdone = bar + 1 + NS;
    uint32_t *holder = reinterpret_cast<uint32_t *>(bar + NBAR);
    __shared__ int s_err;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * TM;
    const int64_t r_begin = (int64_t)blockIdx.y * a.rows_per_split;
    const int64_t r_end = min(a.n, r_begin + a.rows_per_split);
    const int ntiles = r_end > r_begin ? (int)((r_end - r_begin + TN - 1) / TN) : 0;

    if (tid == 0) {
        s_err = 0;
        for (int i = 0; i < NBAR; i++) mbar_init(bar + i, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int j = 0; j < KC; j++) {
        ld[j * TM + tid] = INFINITY;
        li[j * TM + tid] = kEmpty;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *holder;
    float thr = INFINITY;

    auto load_b = [&](int t) {  // tile t into stage t % NS
        uint8_t *dst = sB + (t % NS) * B_STAGE;
        const int y = (int)(r_begin + (int64_t)t * TN);
        mbar_expect_tx(bar + 1 + t % NS, B_STAGE);
        tma_load_2d(dst, &tmB, 0, y, bar + 1 + t % NS);
        tma_load_2d(dst + B_STAGE / 2, &tmB, 64, y, bar + 1 + t % NS);
    };
    auto issue_mma = [&](int t) {  // tile t: stage t % NS, TMEM half t & 1
        const uint8_t *b = sB + (t % NS) * B_STAGE;
        const uint32_t d = tmem + (uint32_t)((t & 1) * TN);
#pragma unroll
        for (int kb = 0; kb < 2; kb++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                mma_bf16(d, sw128_desc(sA + kb * (A_BYTES / 2) + j * 32), sw128_desc(b + kb * (B_STAGE / 2) + j * 32),
                         (kb | j) != 0);
        mma_commit(mdone + (t & 1));
    };

    if (tid == 0 && ntiles > 0) {
        mbar_expect_tx(bar, A_BYTES);
        tma_load_2d(sA, &tmA, 0, (int)q0, bar);
        tma_load_2d(sA + A_BYTES / 2, &tmA, 64, (int)q0, bar);
        for (int t = 0; t < NS && t < ntiles; t++) load_b(t);
        if (wait_bar(bar, 0) && wait_bar(bar + 1, 0)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            issue_mma(0);
        } else {
            s_err = 1;
        }
    }
    __syncthreads();

    for (int t = 0; t < ntiles && !s_err; t++) {
        if (tid == 0 && t + 1 < ntiles) {
            if (wait_bar(bar + 1 + (t + 1) % NS, ((t + 1) / NS) & 1)) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                issue_mma(t + 1);
            } else {
                s_err = 1;
            }
        }
        if (!wait_bar(mdone + (t & 1), (t >> 1) & 1)) s_err = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!s_err) {
            const int64_t col0 = r_begin + (int64_t)t * TN;
            const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((t & 1) * TN);
            for (int c0 = 0; c0 < TN; c0 += 32) {
                uint32_t v[32];
                TMEM_LD32(tbase + c0, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; j++) {
                    const int64_t col = col0 + c0 + j;
                    if (col >= r_end) continue;
                    const float s = __uint_as_float(v[j]);
                    const float dist = a.metric == SVF_IP ? -s : fmaf(-2.f, s, __ldg(a.norms + col));
                    if (dist < thr) {
                        int p = KC - 1;
                        while (p > 0 && ld[(p - 1) * TM + tid] > dist) {
                            ld[p * TM + tid] = ld[(p - 1) * TM + tid];
                            li[p * TM + tid] = li[(p - 1) * TM + tid];
                            p--;
                        }
                        ld[p * TM + tid] = dist;
                        li[p * TM + tid] = (uint32_t)col;
                        thr = ld[(KC - 1) * TM + tid];
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0 && t + NS < ntiles && !s_err) load_b(t + NS);  // stage t % NS is free: MMA t has completed
    }
    if (s_err && tid == 0) set_error(a.status, SVF_ETIMEOUT, blockIdx.x);
    const int64_t q = q0 + tid;
    if (q < a.nq) {
        float *od = a.cand_d + (q * a.splits + blockIdx.y) * KC;
        uint32_t *oi = a.cand_i + (q * a.splits + blockIdx.y) * KC;
        for (int j = 0; j < KC; j++) {
            od[j] = ld[j * TM + tid];
            oi[j] = li[j * TM + tid];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// fp32 rows -> bf16 rows padded to KP columns (+ squared norms).
__global__ void to_bf16_kernel(const float *X, int64_t n, int d, __nv_bfloat16 *out, float *norms) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    float ss = 0.f;
    for (int c = lane; c < KP; c += 32) {
        const float v = c < d ? X[r * d + c] : 0.f;
        out[r * KP + c] = __float2bfloat16_rn(v);
        ss = fmaf(v, v, ss);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) ss += __shfl_xor_sync(kFull, ss, m);
    if (lane == 0 && norms) norms[r] = ss;
}

__global__ void max_kernel(const float *v, int64_t n, unsigned int *out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, s));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}

// Warp per query: exact fp32 distances of all candidates, best k by
// (distance, id), and the certificate (flag = 1 when it fails).
__global__ void rescore_kernel(const float *X, const float *Q, int d, int metric, const float *norms,
                               const unsigned int *maxnorm2, int splits, const float *cand_d, const uint32_t *cand_i,
                               int64_t nq, int k, uint64_t *out_keys, int32_t *flagged, unsigned long long *nflag) {
    extern __shared__ uint64_t rk[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (q >= nq) return;
    const int nc = splits * KC;
    uint64_t *keys = rk + (size_t)wib * nc;
    const float *qr = Q + q * d;
    float qn = 0.f;
    for (int c = lane; c < d; c += 32) qn = fmaf(qr[c], qr[c], qn);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) qn += __shfl_xor_sync(kFull, qn, m);
    float bound = INFINITY;  // smallest per-slice 48th approximate distance
    for (int s = 0; s < splits; s++) bound = fminf(bound, cand_d[(q * splits + s) * KC + KC - 1]);
    for (int e = lane; e < nc; e += 32) {
        const uint32_t id = cand_i[q * nc + e];
        if (id == kEmpty) {
            keys[e] = kPad;
            continue;
        }
        const float *xr = X + (int64_t)id * d;
        float acc = 0.f;
        if (metric == SVF_IP) {
            for (int c = 0; c < d; c++) acc = fmaf(qr[c], xr[c], acc);
            acc = -acc;
        } else {
            for (int c = 0; c < d; c++) {
                const float df = qr[c] - xr[c];
                acc = fmaf(df, df, acc);
            }
        }
        keys[e] = make_key(fkey(acc), id);
    }
    __syncwarp();
    // rank sort of the nc keys (each lane places its own)
    for (int e = lane; e < nc; e += 32) {
        const uint64_t ke = keys[e];
        if (key_is_pad(ke)) continue;
        int pos = 0;
        for (int f = 0; f < nc; f++) pos += keys[f] < ke;
        if (pos < k) out_keys[q * k + pos] = ke;
    }
    int nreal = 0;
    for (int e = lane; e < nc; e += 32) nreal += !key_is_pad(keys[e]);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) nreal += __shfl_xor_sync(kFull, nreal, m);
    for (int e = nreal + lane; e < k; e += 32) out_keys[q * k + e] = kPad;
    __syncwarp();
    if (lane == 0) {
        // certificate: a row outside every slice's candidates has approx
        // distance >= bound, exact >= bound - eps
        const float c = 0.0085f * (metric == SVF_L2 ? 2.f : 1.f);
        const float eps = c * sqrtf(qn) * sqrtf(__uint_as_float(*maxnorm2));
        const float dk = k <= nreal ? fkey_inv((uint32_t)(out_keys[q * k + k - 1] >> 32)) : INFINITY;
        // L2 distances above carry no ||q||^2: add it to the approximate bound
        const float b = metric == SVF_L2 ? bound + qn : bound;
        if (!(b - eps > dk) && isfinite(bound)) {
            const unsigned long long p = atomicAdd(nflag, 1ull);
            flagged[p] = (int32_t)q;
        }
    }
}

__global__ void gather_rows_kernel(const float *Q, int d, const int32_t *idx, int64_t m, float *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * d) return;
    out[i] = Q[(int64_t)idx[i / d] * d + i % d];
}

__global__ void scatter_keys_kernel(const uint64_t *keys, const int32_t *idx, int64_t m, int k, uint64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * k) return;
    out[(int64_t)idx[i / k] * k + i % k] = keys[i];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *m, void *base, int64_t rows, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)KP, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)KP * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

int split_count(int64_t n, int64_t nq) {
    const int64_t qt = (nq + TM - 1) / TM;
    int64_t s = (4 * 148 + qt - 1) / qt;
    const int64_t max_s = (n + TN - 1) / TN;
    if (s > max_s) s = max_s;
    if (s > 64) s = 64;
    return (int)(s < 1 ? 1 : s);
}

struct TcLayout {
    size_t xb, qb, norms, maxn, cd, ci, keys, flagged, nflag, gq, gk, total;
};

TcLayout tc_layout(int64_t n, int64_t nq, int k, int d) {
    TcLayout L{};
    const int s = split_count(n, nq);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.xb = take((size_t)n * KP * 2);
    L.qb = take((size_t)nq * KP * 2);
    L.norms = take((size_t)n * 4);
    L.maxn = take(256);
    L.cd = take((size_t)nq * s * KC * 4);
    L.ci = take((size_t)nq * s * KC * 4);
    L.keys = take((size_t)nq * k * 8);
    L.flagged = take((size_t)nq * 4);
    L.nflag = take(256);
    L.gq = take((size_t)nq * d * 4);
    L.gk = take((size_t)nq * k * 8);
    L.total = o;
    return L;
}

}  // namespace
}  // namespace svf

using namespace svf;

extern "C" {

size_t svf_knn_tc_scratch_bytes(int64_t n, int64_t nq, int32_t d, int32_t k) {
    return tc_layout(n, nq, k, d).total;
}

int svf_knn_tc(const float *X, int64_t n, int32_t d, int32_t metric, const float *Q, int64_t nq, int32_t k,
               void *scratch, size_t scratch_bytes, uint32_t *out_ids, float *out_dist, int64_t *out_fallback,
               void *stream) {
    if (n < 1 || nq < 0 || d < 16 || d > KP || d % 16 || k < 1 || k > 32)
        return fail(SVF_EINVAL, "svf_knn_tc: need n >= 1, 16 <= d <= 128 (multiple of 16), 1 <= k <= 32");
    if (metric != SVF_L2 && metric != SVF_IP) return fail(SVF_EINVAL, "bad metric");
    if (n >= (1ll << 31)) return fail(SVF_EINVAL, "n too large for the tile coordinates");
    if (nq == 0) return SVF_OK;
    if (!X || !Q || !out_ids || !scratch) return fail(SVF_EINVAL, "null pointers");
    const TcLayout L = tc_layout(n, nq, k, d);
    if (scratch_bytes < L.total) return fail(SVF_EINVAL, "scratch of %zu bytes, need %zu", scratch_bytes, L.total);
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *S = reinterpret_cast<uint8_t *>(scratch);
    auto *xb = reinterpret_cast<__nv_bfloat16 *>(S + L.xb);
    auto *qb = reinterpret_cast<__nv_bfloat16 *>(S + L.qb);
    float *norms = reinterpret_cast<float *>(S + L.norms);
    unsigned int *maxn = reinterpret_cast<unsigned int *>(S + L.maxn);
    float *cd = reinterpret_cast<float *>(S + L.cd);
    uint32_t *ci = reinterpret_cast<uint32_t *>(S + L.ci);
    uint64_t *keys = reinterpret_cast<uint64_t *>(S + L.keys);
    int32_t *flagged = reinterpret_cast<int32_t *>(S + L.flagged);
    unsigned long long *nflag = reinterpret_cast<unsigned long long *>(S + L.nflag);
    to_bf16_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(X, n, d, xb, norms);
    to_bf16_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, st>>>(Q, nq, d, qb, nullptr);
    CUDA_TRY(cudaMemsetAsync(maxn, 0, 4, st));
    CUDA_TRY(cudaMemsetAsync(nflag, 0, 8, st));
    max_kernel<<<296, 256, 0, st>>>(norms, n, maxn);
    CUtensorMap ta, tb;
    if (!make_map(&ta, qb, nq, TM) || !make_map(&tb, xb, n, TN))
        return fail(SVF_ECUDA, "cuTensorMapEncodeTiled is unavailable or rejected the layout");
    TcArgs a{};
    a.n = n;
    a.nq = nq;
    a.splits = split_count(n, nq);
    a.rows_per_split = ((n + a.splits - 1) / a.splits + TN - 1) / TN * TN;
    a.metric = metric;
    a.norms = norms;
    a.cand_d = cd;
    a.cand_i = ci;
    // the status word of a stand-alone call lives in the flag counter's slot
    unsigned long long *status = nflag + 8;
    CUDA_TRY(cudaMemsetAsync(status, 0, 8, st));
    a.status = status;
    CUDA_TRY(cudaFuncSetAttribute(tc_knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    dim3 grid((unsigned)((nq + TM - 1) / TM), (unsigned)a.splits);
    tc_knn_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(ta, tb, a);
    CUDA_TRY(cudaGetLastError());
    const int wpb = 4;
    const size_t rsm = (size_t)wpb * a.splits * KC * 8;
    CUDA_TRY(cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    rescore_kernel<<<(unsigned)((nq + wpb - 1) / wpb), wpb * 32, rsm, st>>>(X, Q, d, metric, norms, maxn, a.splits, cd,
                                                                          ci, nq, k, keys, flagged, nflag);
    CUDA_TRY(cudaGetLastError());
    unsigned long long hf[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(&hf[0], nflag, 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&hf[1], status, 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hf[1]) return fail(SVF_ETIMEOUT, "svf_knn_tc: a pipeline wait gave up");
    const int64_t m = (int64_t)hf[0];
    if (m > 0) {
        // queries whose certificate failed: exact SIMT scan
        float *gq = reinterpret_cast<float *>(S + L.gq);
        uint64_t *gk = reinterpret_cast<uint64_t *>(S + L.gk);
        gather_rows_kernel<<<(unsigned)((m * d + 255) / 256), 256, 0, st>>>(Q, d, flagged, m, gq);
        KnnArgs ka{};
        ka.X.base = reinterpret_cast<const uint8_t *>(X);
        ka.X.pitch = (int64_t)d * 4;
        ka.X.nchunk = d / 4;
        ka.X.d = d;
        ka.X.dtype = SVF_F32;
        ka.X.metric = metric;
        ka.X.copy_bytes = d * 4;
        ka.n = n;
        ka.Q = gq;
        ka.q_row_bytes = d * 4;
        ka.nq = m;
        ka.self_base = -1;
        ka.k = k;
        ka.out_keys = gk;
        CUDA_TRY(launch_knn(ka, st));
        scatter_keys_kernel<<<(unsigned)((m * k + 255) / 256), 256, 0, st>>>(gk, flagged, m, k, keys);
    }
    CUDA_TRY(launch_keys_to_out(keys, nq, k, k, SVF_F32, metric, out_ids, reinterpret_cast<uint32_t *>(out_dist), st));
    if (out_fallback) *out_fallback = m;
    return SVF_OK;
}

}  // extern "C"
