// tc_knn.cu -- exact brute-force k nearest neighbours on the tensor cores
// (ground truth, Sec. 6.1 "exhaustive linear scan"), for fp32 stores with
// d <= 128.
//
// 1. Rows and queries are rounded to bf16, zero-padded to a multiple of 32
//    columns (one 64-byte swizzle atom per 32 columns).
// 2. tc_knn_kernel: a CTA owns 128 queries and one slice of the database,
//    in a warp-specialised pipeline linked by mbarriers.  A producer warp
//    TMA-loads 256-row database tiles into a ring of shared-memory stages;
//    an MMA warp issues tcgen05.mma (kind::f16, bf16 in, fp32 accumulate,
//    M=128, N=256, K=16) for each tile into one of two TMEM accumulator
//    buffers; eight epilogue warps (two per TMEM lane group, one per column
//    half) read a buffer with tcgen05.ld, release it, and keep each query's
//    16 best approximate distances per half: a max tree over 32 columns
//    tests them against the lane's current 16th, and only when a lane of
//    the warp beats it are the passing columns appended to a pending buffer
//    and merged, all lanes at once, into the sorted lists.  For large sets a
//    first pass of the same kernel over every 32nd tile gives each query a
//    starting threshold (its 16th best in that sample), so the lists start
//    near their final values and few chunks take the append path.
// 3. rescore_kernel: per query, the candidates of all lists get exact fp32
//    distances and the best k by (distance, id) are kept.  A certificate
//    checks the result: every row left out of a list has an approximate
//    distance at least that list's 16th, and the bf16 error of a distance is
//    at most c ||q|| ||x|| (two roundings of 2^-8 each per product, plus the
//    fp32 sums; c = 0.0085 covers d <= 128, doubled for L2), so
//    if min_list(16th) - eps exceeds the k-th exact distance no row can be
//    missing.  Queries that fail it are recomputed by the SIMT kernel
//    (knn.cu).
// 4. The build (tc_build_knn): the rows are their own queries, in chunks of
//    131,072; band_rescore_kernel re-scores only the candidates within the
//    error band of the 2R-th and certifies them the same way; the rows that
//    fail are gathered across chunks and rescanned by the SIMT kernel.  For
//    uint8 stores the bf16 copies are exact and every partial sum of the
//    products is an integer below 2^24, so the scan's distances are exact,
//    the band has no error margin and the re-scoring is in int32.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "index_impl.h"

namespace svf {
namespace {

constexpr int TM = 128, TN = 256, KP = 128;   // KP: largest padded dimension
constexpr int KA = 32;                         // columns per 64-byte swizzle atom
constexpr int HALVES = 2;                      // epilogue warps per TMEM lane group (column halves)
constexpr int KC = 16;                         // candidates kept per (query, slice, half)
constexpr int EPI_WARPS = 4 * HALVES;          // warps 0-7: epilogue; warp w reads lanes 32 (w % 4) ..
constexpr int THREADS = (EPI_WARPS + 2) * 32;  // warp 8: TMA producer, warp 9: MMA issuer
constexpr int NS_MAX = 8;                      // database tile stages in shared memory (as many as fit)
constexpr int NT = 2;                          // accumulator buffers of TN columns in TMEM
constexpr int BUF = 16;                        // pending candidates of one 16-column sub-chunk
constexpr int A_ATOM = TM * KA * 2, B_ATOM = TN * KA * 2;
constexpr int LIST_BYTES = HALVES * KC * TM * 8;
constexpr int BUF_BYTES = HALVES * BUF * TM * 8;
constexpr int NBAR = 1 + 2 * NS_MAX + 2 * NT;  // A; full/empty per stage; full/empty per TMEM buffer
constexpr int BAR_BYTES = 1024;                 // barriers + TMEM address, rounded to keep B aligned
static_assert(8 * NBAR + 4 <= BAR_BYTES, "barrier area");
constexpr int SMEM_LIMIT = 232448;              // opt-in shared memory per block
// layout: [align pad][A: TM x kp][lists][pending][barriers][ns stages of TN x kp]
__host__ __device__ constexpr int smem_fixed(int kp) { return 1024 + TM * kp * 2 + LIST_BYTES + BUF_BYTES + BAR_BYTES; }
__host__ __device__ constexpr int stage_bytes(int kp) { return TN * kp * 2; }
static_assert(smem_fixed(KP) + 2 * stage_bytes(KP) <= SMEM_LIMIT, "two stages at the largest width");
// Error bound of a bf16 product sum: each operand is rounded to bf16 (8-bit
// significand, relative error <= 2^-8), so each product is off by at most
// (2^-7 + 2^-16) |q_i x_i|, and the fp32 accumulation of d <= 128 products
// adds at most about d 2^-23 of their magnitude: |error| <= c ||q|| ||x||
// with c = 0.0079 for inner products; 0.0085 keeps a margin above that (the
// squared-L2 form, -2 q.x, doubles it).
constexpr float kBf16ErrC = 0.0085f;
constexpr int64_t kTcBuildMinRows = 1 << 16;  // smaller builds take the SIMT scan
constexpr int kSeedStride = 64;            // seed pass reads one tile in 64
constexpr int kSeedRank = 8;               // seed = 8th best of the sample (~512th of all rows)
constexpr int64_t kSeedMinRows = 1 << 17;  // smaller sets skip the seed pass
static_assert(kSeedRank <= HALVES * KC, "seed rank within the sample lists");
constexpr uint32_t kTmemCols = NT * TN;
static_assert(kTmemCols <= 512, "TMEM columns");

struct TcArgs {
    int64_t n, nq;
    int64_t rows_per_split;
    int splits;
    int metric;
    int atoms;           // padded dimension / KA
    int ns;              // stages in the ring
    int tile_stride;     // 1, or s > 1: every s-th tile only (the seed pass)
    const float *seed;   // [nq] starting threshold per query, or null (+inf)
    const float *norms;  // ||x||^2 (L2)
    float *cand_d;       // [nq][splits][HALVES][KC]
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

// UMMA shared-memory descriptor: K-major operand, 64-byte swizzle (rows of
// 32 bf16), 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    return ((addr >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
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

// max of 32 floats (as bit patterns) by a pairwise tree
__device__ __forceinline__ float max32(const uint32_t *v) {
    float m[16];
#pragma unroll
    for (int i = 0; i < 16; i++) m[i] = fmaxf(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; i++) m[i] = fmaxf(m[i], m[i + w]);
    return m[0];
}

// -(min of 32 floats)
__device__ __forceinline__ float max32_neg(const uint32_t *v) {
    float m[16];
#pragma unroll
    for (int i = 0; i < 16; i++) m[i] = fminf(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; i++) m[i] = fminf(m[i], m[i + w]);
    return -m[0];
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

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Warp-specialised pipeline, linked by mbarriers (no block-wide barrier in
// the loop):
//   producer (warp 8)  TMA: database tile t -> stage t % ns
//   MMA      (warp 9)  tile t x query tile -> TMEM buffer t % NT
//   epilogue (0-7)     TMEM buffer -> registers, release the buffer, then
//                      filter / append / merge into the per-query lists.
__global__ void __launch_bounds__(THREADS, 1)
    tc_knn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
    extern __shared__ uint8_t sm_raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~(uintptr_t)1023);
    const int ns = a.ns;
    const uint32_t a_atom = (uint32_t)A_ATOM, b_atom = (uint32_t)B_ATOM, b_stage = (uint32_t)(a.atoms * B_ATOM);
    uint8_t *sA = sm;
    float *ld = reinterpret_cast<float *>(sm + a.atoms * A_ATOM);
    uint32_t *li = reinterpret_cast<uint32_t *>(ld + HALVES * KC * TM);
    float2 *buf = reinterpret_cast<float2 *>(li + HALVES * KC * TM);  // [HALVES][BUF][TM] pending (distance, row)
    uint64_t *barA = reinterpret_cast<uint64_t *>(buf + HALVES * BUF * TM);
    uint64_t *full = barA + 1, *empty = full + NS_MAX;       // stage s loaded / consumed by the MMA
    uint64_t *tfull = empty + NS_MAX, *tempty = tfull + NT;  // TMEM buffer b accumulated / read out
    uint32_t *holder = reinterpret_cast<uint32_t *>(tempty + NT);
    uint8_t *sB = reinterpret_cast<uint8_t *>(barA) + BAR_BYTES;
    __shared__ int s_err, s_nl, s_nc, s_nm;
    volatile int *err = &s_err;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qr = tid & (TM - 1), half = (tid >> 7) & (HALVES - 1);  // epilogue: query row, column half
    float *lst_d = ld + half * KC * TM + qr;  // this thread's list, stride TM
    uint32_t *lst_i = li + half * KC * TM + qr;
    float2 *pend = buf + half * BUF * TM + qr;
    const int64_t q0 = (int64_t)blockIdx.x * TM;
    const int64_t r_begin = (int64_t)blockIdx.y * a.rows_per_split;
    const int64_t r_end = min(a.n, r_begin + a.rows_per_split);
    const int64_t span = (int64_t)TN * a.tile_stride;  // rows from one tile to the next
    const int ntiles = r_end > r_begin ? (int)((r_end - r_begin + span - 1) / span) : 0;

    if (tid == 0) {
        s_err = 0;
        s_nl = s_nc = s_nm = 0;
        mbar_init(barA, 1);
        for (int i = 0; i < ns; i++) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        for (int i = 0; i < NT; i++) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, EPI_WARPS);
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // A list starts full of (seed, empty) entries: rows at or above the seed
    // are never kept, and the list's KC-th value never exceeds the seed.
    const float seed0 = (a.seed && q0 + qr < a.nq) ? a.seed[q0 + qr] : INFINITY;
    if (warp < EPI_WARPS)
        for (int j = 0; j < KC; j++) {
            lst_d[j * TM] = seed0;
            lst_i[j * TM] = kEmpty;
        }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *holder;

    if (warp == EPI_WARPS) {
        // ---------------------------------------------------------- producer
        if (lane == 0 && ntiles > 0) {
            mbar_expect_tx(barA, (uint32_t)a.atoms * a_atom);
            for (int at = 0; at < a.atoms; at++) tma_load_2d(sA + at * a_atom, &tmA, at * KA, (int)q0, barA);
            int nl = 0, st = 0;
            uint32_t ph = 0;
            for (int t = 0; t < ntiles && !*err; t++) {
                if (!wait_bar(empty + st, ph ^ 1)) {  // round 0 passes at once
                    *err = 1;
                    break;
                }
                const int y = (int)(r_begin + (int64_t)t * span);
                mbar_expect_tx(full + st, b_stage);
                for (int at = 0; at < a.atoms; at++)
                    tma_load_2d(sB + st * b_stage + at * b_atom, &tmB, at * KA, y, full + st);
                nl = t + 1;
                if (++st == ns) {
                    st = 0;
                    ph ^= 1;
                }
            }
            s_nl = nl;
        }
    } else if (warp == EPI_WARPS + 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0 && ntiles > 0) {
            int nc = 0, nm = 0, st = 0;
            uint32_t ph = 0;
            if (!wait_bar(barA, 0)) *err = 1;
            for (int t = 0; t < ntiles && !*err; t++) {
                const int b = t % NT;
                if (!wait_bar(full + st, ph)) {
                    *err = 1;
                    break;
                }
                nc = t + 1;
                if (!wait_bar(tempty + b, ((t / NT) & 1) ^ 1)) {
                    *err = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint8_t *bs = sB + st * b_stage;
                const uint32_t d = tmem + (uint32_t)(b * TN);
                for (int at = 0; at < a.atoms; at++)
#pragma unroll
                    for (int j = 0; j < 2; j++)  // K = 16 per MMA: two per atom
                        mma_bf16(d, sw64_desc(sA + at * a_atom + j * 32), sw64_desc(bs + at * b_atom + j * 32),
                                 (at | j) != 0);
                mma_commit(empty + st);  // the stage may be refilled once these MMAs have read it
                mma_commit(tfull + b);
                nm = t + 1;
                if (++st == ns) {
                    st = 0;
                    ph ^= 1;
                }
            }
            s_nc = nc;
            s_nm = nm;
        }
    } else {
        // ---------------------------------------------------------- epilogue
        float thr = seed0;  // this query's KC-th best approximate distance so far
        int cnt = 0;           // pending entries
        // Merge the pending entries into the sorted list.  All lanes of a
        // warp merge together (each its own query), so the insertions run
        // side by side instead of one lane at a time; rows past the slice
        // end (zero fill of the last tile) are dropped here.
        auto flush = [&]() {
            for (int e = 0; e < cnt; e++) {
                const float2 c = pend[e * TM];
                const uint32_t col = __float_as_uint(c.y);
                if (c.x < thr && (int64_t)col < r_end) {
                    int p = KC - 1;
                    while (p > 0 && lst_d[(p - 1) * TM] > c.x) {
                        lst_d[p * TM] = lst_d[(p - 1) * TM];
                        lst_i[p * TM] = lst_i[(p - 1) * TM];
                        p--;
                    }
                    lst_d[p * TM] = c.x;
                    lst_i[p * TM] = col;
                    thr = lst_d[(KC - 1) * TM];
                }
            }
            cnt = 0;
        };
        for (int t = 0; t < ntiles; t++) {
            const int b = t % NT;
            const bool got = wait_bar(tfull + b, (t / NT) & 1);
            if (__any_sync(kFull, !got || *err)) {  // warp-uniform exit
                if (lane == 0) *err = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            constexpr int NC = TN / HALVES;         // columns of this warp
            constexpr int NG = NC < 64 ? NC : 64;  // columns read from TMEM at a time
            const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(b * TN + half * NC);
            const int64_t col0 = r_begin + (int64_t)t * span + half * NC;
#pragma unroll 1
            for (int g = 0; g < NC; g += NG) {
                uint32_t v[NG];
#pragma unroll
                for (int c = 0; c < NG; c += 32) TMEM_LD32(tbase + g + c, (v + c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (g + NG == NC) {  // all of this warp's columns are in registers: free the buffer
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty + b);
                }
#pragma unroll
                for (int c0 = 0; c0 < NG; c0 += 32) {
                    const uint32_t cb = (uint32_t)(col0 + g + c0);
                    if (a.metric != SVF_IP) {
                        // L2 without ||q||^2: lane j holds the norm of column j
                        const float nrm = __ldg(a.norms + min((int64_t)cb + lane, a.n - 1));
#pragma unroll
                        for (int j = 0; j < 32; j++)
                            v[c0 + j] =
                                __float_as_uint(fmaf(-2.f, __uint_as_float(v[c0 + j]), __shfl_sync(kFull, nrm, j)));
                    }
                    // smallest approximate distance of the 32 columns; the
                    // append path runs only when some lane of the warp beats
                    // its threshold
                    const float dmin = a.metric == SVF_IP ? -max32(v + c0) : -max32_neg(v + c0);
                    if (__any_sync(kFull, dmin < thr)) {
#pragma unroll
                        for (int h16 = 0; h16 < 32; h16 += BUF) {
#pragma unroll
                            for (int j = h16; j < h16 + BUF; j++) {
                                const float dist =
                                    a.metric == SVF_IP ? -__uint_as_float(v[c0 + j]) : __uint_as_float(v[c0 + j]);
                                if (dist < thr) pend[(cnt++) * TM] = make_float2(dist, __uint_as_float(cb + j));
                            }
                            flush();
                        }
                    }
                }
            }
        }

    }
    __syncthreads();
    if (s_err && tid == 0) {
        // drain: copies and MMAs still in flight land before TMEM is freed
        if (ntiles > 0) wait_bar(barA, 0);
        for (int t = s_nc; t < s_nl; t++) wait_bar(full + t % ns, (t / ns) & 1);
        if (s_nm > 0) wait_bar(tfull + (s_nm - 1) % NT, ((s_nm - 1) / NT) & 1);  // commits track all earlier MMAs
        set_error(a.status, SVF_ETIMEOUT, blockIdx.x);
    }
    const int64_t q = q0 + qr;
    if (warp < EPI_WARPS && q < a.nq) {
        const int64_t o = ((q * a.splits + blockIdx.y) * HALVES + half) * KC;
        for (int j = 0; j < KC; j++) {
            a.cand_d[o + j] = lst_d[j * TM];
            a.cand_i[o + j] = lst_i[j * TM];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// fp32 rows -> bf16 rows padded to kp columns (+ squared norms).
__global__ void to_bf16_kernel(const float *X, int64_t n, int d, int kp, __nv_bfloat16 *out, float *norms) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    float ss = 0.f;
    for (int c = lane; c < kp; c += 32) {
        const float v = c < d ? X[r * d + c] : 0.f;
        out[r * kp + c] = __float2bfloat16_rn(v);
        ss = fmaf(v, v, ss);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) ss += __shfl_xor_sync(kFull, ss, m);
    if (lane == 0 && norms) norms[r] = ss;
}

// uint8 rows -> bf16 rows padded to kp columns (+ squared norms).  Every
// value 0..255 is exact in bf16, and for d <= 128 every product and every sum
// of them is an integer below 2^24, so the tensor-core pass computes the exact
// distances in fp32.
__global__ void u8_to_bf16_kernel(const uint8_t *X, int64_t n, int d, int kp, __nv_bfloat16 *out, float *norms) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    uint32_t ss = 0;
    for (int c = lane; c < kp; c += 32) {
        const uint32_t v = c < d ? X[r * d + c] : 0u;
        out[r * kp + c] = __float2bfloat16_rn((float)v);
        ss += v * v;
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) ss += __shfl_xor_sync(kFull, ss, m);
    if (lane == 0 && norms) norms[r] = (float)ss;
}

__global__ void max_kernel(const float *v, int64_t n, unsigned int *out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, s));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}

// Seed of a query: the r-th smallest approximate distance in the union of
// its sorted lists from the strided sample pass (r rounds of taking the
// smallest list head).
__global__ void seed_kernel(const float *cand_d, int64_t nq, int lists, int r, float *seed) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const float *l = cand_d + q * lists * KC;
    uint8_t head[64 * HALVES];
    for (int i = 0; i < lists; i++) head[i] = 0;
    float v = INFINITY;
    for (int m = 0; m < r; m++) {
        int best = -1;
        float bv = INFINITY;
        for (int i = 0; i < lists; i++)
            if (head[i] < KC && l[i * KC + head[i]] < bv) {
                bv = l[i * KC + head[i]];
                best = i;
            }
        if (best < 0) break;
        v = bv;
        head[best]++;
    }
    seed[q] = v;
}

// Warp per query: exact fp32 distances of all candidates, best k by
// (distance, id), and the certificate (flag = 1 when it fails).
__global__ void rescore_kernel(const float *X, const float *Q, int d, int metric, const float *norms,
                               const unsigned int *maxnorm2, int lists, const float *cand_d, const uint32_t *cand_i,
                               int64_t nq, int k, uint64_t *out_keys, int32_t *flagged, unsigned long long *nflag) {
    extern __shared__ uint64_t rk[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (q >= nq) return;
    const int nc = lists * KC;
    uint64_t *keys = rk + (size_t)wib * nc;
    const float *qr = Q + q * d;
    float qn = 0.f;
    for (int c = lane; c < d; c += 32) qn = fmaf(qr[c], qr[c], qn);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) qn += __shfl_xor_sync(kFull, qn, m);
    float bound = INFINITY;  // smallest KC-th approximate distance over the lists
    for (int s = 0; s < lists; s++) bound = fminf(bound, cand_d[(q * lists + s) * KC + KC - 1]);
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
        const float c = kBf16ErrC * (metric == SVF_L2 ? 2.f : 1.f);
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

// Exact K nearest neighbours from the candidate lists when K is large (the
// build's 2R): warp per query.  The candidates (lists x KC <= 32 NPL, the
// query's own row excluded for a self join) are sorted by their approximate
// distance a(x); only the band a(x) <= a_K + 2 eps is re-scored exactly, a_K
// being the K-th smallest approximate distance: each of the K candidates
// with a(x) <= a_K has exact distance <= a_K + eps, so the K-th exact
// distance D_K <= a_K + eps, and a candidate outside the band has exact
// distance > a_K + eps >= D_K.  The list certificate is the one of
// rescore_kernel (rows outside every list have approximate distance >= the
// smallest list bound); a query that fails it, or has fewer than K
// candidates, is flagged for the exact SIMT scan.
//
// Query q is row q0 + q of the store, or row qids[q] when qids is set (the
// second pass over the rows whose certificate failed).
//
// U8 (a uint8 store): the approximate distances are exact (u8_to_bf16_kernel),
// so eps_c is 0, the band is the candidates at or below a_K, the exact
// distances are integers (the store's keys: squared L2, or -dot through the
// order-preserving map) and the certificate is that the smallest list bound
// exceeds D_K strictly (a row left out of every list with the same distance
// could precede the K-th by id).
template <int NPL, bool U8>
__global__ void band_rescore_kernel(const void *Xv, int d, int metric, const unsigned int *maxnorm2, int lists,
                                    const float *cand_d, const uint32_t *cand_i, int64_t q0, int64_t nq, int K,
                                    float eps_c, uint64_t *out_keys, int32_t *flagged, unsigned long long *nflag,
                                    const int64_t *qids) {
    extern __shared__ float4 bq[];  // per warp: the query row (d <= 128 floats, or d bytes)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (q >= nq) return;
    const int nc = lists * KC;
    const int64_t qrow = qids ? qids[q] : q0 + q;  // the query's own row of the store
    const uint32_t self = (uint32_t)qrow;
    const float *X = reinterpret_cast<const float *>(Xv);
    const uint8_t *X8 = reinterpret_cast<const uint8_t *>(Xv);
    float4 *qs = bq + wib * (KP / 4);
    float qn = 0.f;
    if constexpr (U8) {
        const uint4 *qr8 = reinterpret_cast<const uint4 *>(X8 + qrow * d);
        uint4 *qs8 = reinterpret_cast<uint4 *>(qs);
        for (int c = lane; c < d / 16; c += 32) qs8[c] = qr8[c];
        __syncwarp();
        uint32_t qi = 0;
        for (int c = lane; c < d; c += 32) {
            const uint32_t v = X8[qrow * d + c];
            qi += v * v;
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) qi += __shfl_xor_sync(kFull, qi, m);
        qn = (float)qi;
    } else {
        const float *qr = X + qrow * d;
        for (int c = lane; c < d / 4; c += 32) qs[c] = reinterpret_cast<const float4 *>(qr)[c];
        __syncwarp();
        for (int c = lane; c < d; c += 32) qn = fmaf(qr[c], qr[c], qn);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) qn += __shfl_xor_sync(kFull, qn, m);
    }
    float bound = INFINITY;
    for (int s = lane; s < lists; s += 32) bound = fminf(bound, cand_d[(q * lists + s) * KC + KC - 1]);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) bound = fminf(bound, __shfl_xor_sync(kFull, bound, m));
    uint64_t ak[NPL];
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        const int e = s * 32 + lane;
        const uint32_t id = e < nc ? cand_i[q * nc + e] : kEmpty;
        ak[s] = (id == kEmpty || id == self) ? kPad : make_key(fkey(cand_d[q * nc + e]), id);
    }
    warp_sort<NPL>(ak, lane);
    const float c = eps_c * (metric == SVF_L2 ? 2.f : 1.f);
    const float eps = c * sqrtf(qn) * sqrtf(__uint_as_float(*maxnorm2));
    uint64_t akK = kPad;
#pragma unroll
    for (int s = 0; s < NPL; s++)
        if (s == ((K - 1) >> 5)) akK = shfl64(ak[s], (K - 1) & 31);
    bool fail = key_is_pad(akK);
    int nb = 0;
    if (!fail) {
        const float cut = fkey_inv((uint32_t)(akK >> 32)) + 2.f * eps;
        // the band is a prefix of the sorted candidates
#pragma unroll
        for (int s = 0; s < NPL; s++)
            nb += __popc(__ballot_sync(kFull, !key_is_pad(ak[s]) && fkey_inv((uint32_t)(ak[s] >> 32)) <= cut));
#pragma unroll
        for (int s = 0; s < NPL; s++) {
            const int e = s * 32 + lane;
            uint64_t kx = kPad;
            if (e < nb && U8) {
                // the row in 16-byte loads, exact in int32
                const uint32_t id = key_id(ak[s]);
                const uint4 *xr = reinterpret_cast<const uint4 *>(X8 + (int64_t)id * d);
                const uint4 *qs8 = reinterpret_cast<const uint4 *>(qs);
                uint32_t acc = 0;
#pragma unroll 8
                for (int c = 0; c < d / 16; c++) {
                    const uint4 x = __ldg(xr + c), qv = qs8[c];
                    if (metric == SVF_IP) {
                        acc = __dp4a(x.x, qv.x, acc);
                        acc = __dp4a(x.y, qv.y, acc);
                        acc = __dp4a(x.z, qv.z, acc);
                        acc = __dp4a(x.w, qv.w, acc);
                    } else {
                        const uint32_t a0 = __vabsdiffu4(x.x, qv.x), a1 = __vabsdiffu4(x.y, qv.y),
                                       a2 = __vabsdiffu4(x.z, qv.z), a3 = __vabsdiffu4(x.w, qv.w);
                        acc = __dp4a(a0, a0, acc);
                        acc = __dp4a(a1, a1, acc);
                        acc = __dp4a(a2, a2, acc);
                        acc = __dp4a(a3, a3, acc);
                    }
                }
                kx = make_key(metric == SVF_IP ? ((uint32_t)(-(int32_t)acc) ^ 0x80000000u) : acc, id);
            } else if (e < nb) {
                // the row in 16-byte loads, summed in element order
                const uint32_t id = key_id(ak[s]);
                const float4 *xr = reinterpret_cast<const float4 *>(X + (int64_t)id * d);
                float acc = 0.f;
#pragma unroll 8
                for (int c4 = 0; c4 < d / 4; c4++) {
                    const float4 x = __ldg(xr + c4), qv = qs[c4];
                    if (metric == SVF_IP) {
                        acc = fmaf(qv.x, x.x, acc);
                        acc = fmaf(qv.y, x.y, acc);
                        acc = fmaf(qv.z, x.z, acc);
                        acc = fmaf(qv.w, x.w, acc);
                    } else {
                        acc = fmaf(qv.x - x.x, qv.x - x.x, acc);
                        acc = fmaf(qv.y - x.y, qv.y - x.y, acc);
                        acc = fmaf(qv.z - x.z, qv.z - x.z, acc);
                        acc = fmaf(qv.w - x.w, qv.w - x.w, acc);
                    }
                }
                kx = make_key(fkey(metric == SVF_IP ? -acc : acc), id);
            }
            ak[s] = kx;
        }
        warp_sort<NPL>(ak, lane);
        uint64_t dK = kPad;
#pragma unroll
        for (int s = 0; s < NPL; s++)
            if (s == ((K - 1) >> 5)) dK = shfl64(ak[s], (K - 1) & 31);
        const uint32_t dkk = (uint32_t)(dK >> 32);
        const float DK = !U8 ? fkey_inv(dkk) : metric == SVF_IP ? (float)(int32_t)(dkk ^ 0x80000000u) : (float)dkk;
        const float b = metric == SVF_L2 ? bound + qn : bound;
        fail = key_is_pad(dK) || (!(b - eps > DK) && isfinite(bound));
    }
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        const int e = s * 32 + lane;
        if (e < K) out_keys[q * K + e] = fail ? kPad : ak[s];
    }
    if (fail && lane == 0) {
        const unsigned long long p = atomicAdd(nflag, 1ull);
        flagged[p] = (int32_t)q;
    }
}

__global__ void self_ids_kernel(const int32_t *idx, int64_t m, int64_t q0, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = q0 + idx[i];
}

// Rows X[ids[i]] -> out[i] (fp32, d values each).
__global__ void gather_ids_kernel(const float *X, int d, const int64_t *ids, int64_t m, float *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * d) return;
    out[i] = X[ids[i / d] * d + i % d];
}

// out[i] = ids[idx[i]]: store ids of the flagged entries of an id list.
__global__ void pick_ids_kernel(const int32_t *idx, int64_t m, const int64_t *ids, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = ids[idx[i]];
}

// bf16 rows xb[ids[i]] -> out[i] (kp values each).
__global__ void gather_bf16_kernel(const __nv_bfloat16 *xb, int kp, const int64_t *ids, int64_t m, __nv_bfloat16 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * kp) return;
    out[i] = xb[ids[i / kp] * kp + i % kp];
}

// uint8 rows X[ids[i]] -> out[i] (d bytes each).
__global__ void gather_ids_u8_kernel(const uint8_t *X, int d, const int64_t *ids, int64_t m, uint8_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * d) return;
    out[i] = X[ids[i / d] * d + i % d];
}

// keys[i] (k per row) -> out[ids[i]] (k per row).
__global__ void scatter_ids_kernel(const uint64_t *keys, const int64_t *ids, int64_t m, int k, uint64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * k) return;
    out[ids[i / k] * k + i % k] = keys[i];
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

bool make_map(CUtensorMap *m, void *base, int64_t rows, int kp, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    cuuint32_t box[2] = {KA, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// Database slices per query tile: one CTA per SM, so the grid (query
// tiles x slices) should fill whole waves of the SMs.  Take the
// smallest count that fills at least one wave with >= 95% of the last
// wave busy, else the best fill up to 64 slices.
int split_count(int64_t n, int64_t nq) {
    const int kSMs = sm_count();
    const int64_t qt = (nq + TM - 1) / TM;
    const int64_t max_s = std::min<int64_t>(64, (n + TN - 1) / TN);
    int64_t best = 1;
    double best_eff = 0.0;
    for (int64_t s = 1; s <= max_s; s++) {
        const int64_t ctas = qt * s;
        const double eff = (double)ctas / (double)(kSMs * ((ctas + kSMs - 1) / kSMs));
        if (ctas >= kSMs && eff >= 0.95) return (int)s;
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = s;
        }
    }
    return (int)best;
}

// The approximate pass over bf16 rows xb [n][kp] for bf16 queries qb [nq][kp]:
// a seed pass over every kSeedStride-th tile for large n, then the full pass
// into cand_d / cand_i [nq][2 * splits][KC].  splits: at least min_splits,
// else split_count's choice, at most 64.
struct TcPass {
    const __nv_bfloat16 *xb, *qb;
    int64_t n, nq;
    int kp, metric;
    const float *norms;
    float *cd, *seed;
    uint32_t *ci;
    unsigned long long *status;
    int splits;  // out
};

int tc_pass(TcPass &p, int min_splits, int max_splits, cudaStream_t st) {
    CUtensorMap ta, tb;
    if (!make_map(&ta, const_cast<__nv_bfloat16 *>(p.qb), p.nq, p.kp, TM) ||
        !make_map(&tb, const_cast<__nv_bfloat16 *>(p.xb), p.n, p.kp, TN))
        return fail(SVF_ECUDA, "cuTensorMapEncodeTiled is unavailable or rejected the layout");
    TcArgs a{};
    a.n = p.n;
    a.nq = p.nq;
    a.metric = p.metric;
    a.atoms = p.kp / KA;
    a.norms = p.norms;
    a.cand_d = p.cd;
    a.cand_i = p.ci;
    a.status = p.status;
    a.ns = std::min(NS_MAX, (SMEM_LIMIT - smem_fixed(p.kp)) / stage_bytes(p.kp));
    const int smem = smem_fixed(p.kp) + a.ns * stage_bytes(p.kp);
    CUDA_TRY(cudaFuncSetAttribute(tc_knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const unsigned qtiles = (unsigned)((p.nq + TM - 1) / TM);
    a.splits = std::min(max_splits, std::max(min_splits, split_count(p.n, p.nq)));
    a.rows_per_split = ((p.n + a.splits - 1) / a.splits + TN - 1) / TN * TN;
    a.tile_stride = 1;
    if (p.n >= kSeedMinRows) {
        // Seed pass: every kSeedStride-th tile, one slice (few, long lists:
        // an unseeded list pays for its first insertions).  The r-th best of
        // that sample sits near rank r * kSeedStride of the whole set, a
        // threshold most rows of the full pass then fail at once.
        TcArgs s1 = a;
        s1.splits = 1;
        s1.rows_per_split = (p.n + TN - 1) / TN * TN;
        s1.tile_stride = kSeedStride;
        s1.seed = nullptr;
        tc_knn_kernel<<<dim3(qtiles, 1), THREADS, smem, st>>>(ta, tb, s1);
        CUDA_TRY(cudaGetLastError());
        seed_kernel<<<(unsigned)((p.nq + 127) / 128), 128, 0, st>>>(p.cd, p.nq, HALVES, kSeedRank, p.seed);
        CUDA_TRY(cudaGetLastError());
        a.seed = p.seed;
    }
    tc_knn_kernel<<<dim3(qtiles, (unsigned)a.splits), THREADS, smem, st>>>(ta, tb, a);
    CUDA_TRY(cudaGetLastError());
    p.splits = a.splits;
    return SVF_OK;
}

struct TcLayout {
    size_t xb, qb, norms, maxn, cd, ci, keys, flagged, nflag, gq, gk, seed, total;
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
    const int kp = (d + KA - 1) / KA * KA;
    L.xb = take((size_t)n * kp * 2);
    L.qb = take((size_t)nq * kp * 2);
    L.norms = take((size_t)n * 4);
    L.maxn = take(256);
    L.cd = take((size_t)nq * s * HALVES * KC * 4);
    L.ci = take((size_t)nq * s * HALVES * KC * 4);
    L.keys = take((size_t)nq * k * 8);
    L.flagged = take((size_t)nq * 4);
    L.nflag = take(256);
    L.gq = take((size_t)nq * d * 4);
    L.gk = take((size_t)nq * k * 8);
    L.seed = take((size_t)nq * 4);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------- build
// Slices of the build's scan: 2 * splits lists of KC candidates hold four
// times the K neighbours wanted, so each list's bound lies far beyond them.
constexpr int kBuildNPLMax = 16;  // candidates per lane in band_rescore_kernel: at most 512 per row
int build_splits(int K) { return std::max(1, (4 * K + 2 * KC - 1) / (2 * KC)); }

struct TcBuildLayout {
    size_t xb, norms, maxn, cd, ci, seed, flagged, nflag, gq, gk, gself, gfail, total;
    int64_t chunk;
};

TcBuildLayout tc_build_layout(int64_t n, int d, int K) {
    TcBuildLayout L{};
    const int kp = (d + KA - 1) / KA * KA;
    L.chunk = std::min<int64_t>(std::max<int64_t>(n, 1), 131072);
    const int lists = 2 * build_splits(K);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.xb = take((size_t)n * kp * 2);
    L.norms = take((size_t)n * 4);
    L.maxn = take(256);
    L.cd = take((size_t)L.chunk * lists * KC * 4);
    L.ci = take((size_t)L.chunk * lists * KC * 4);
    L.seed = take((size_t)L.chunk * 4);
    L.flagged = take((size_t)L.chunk * 4);
    L.nflag = take(256);
    L.gq = take((size_t)L.chunk * d * 4);
    L.gk = take((size_t)L.chunk * K * 8);
    L.gself = take((size_t)L.chunk * 8);
    L.gfail = take((size_t)L.chunk * 8);
    L.total = o;
    return L;
}

}  // namespace

// Inner product only: for squared L2 the bound eps grows with ||q|| ||x||,
// which for data far from the origin exceeds the gaps between neighbour
// distances, so the certificate would fail for most rows.
bool tc_build_applies(int dtype, int metric, int d, int64_t n, int K) {
    // fp32: inner product only (the bf16 bound above); uint8: exact for both
    // metrics (d <= 128: every partial sum an integer below 2^24)
    const bool kind = (dtype == SVF_F32 && metric == SVF_IP) || (dtype == SVF_U8 && (metric == SVF_L2 || metric == SVF_IP));
    return kind && d % 16 == 0 && d <= KP && n >= kTcBuildMinRows && K >= 1 &&
           2 * build_splits(K) * KC <= 32 * kBuildNPLMax && n < (1ll << 31);
}

size_t tc_build_scratch_bytes(int64_t n, int d, int K) { return tc_build_layout(n, d, K).total; }

// Exact K nearest neighbours (self excluded) of every row of an fp32 store,
// sorted by (distance, id): the tensor-core scan of the rows against
// themselves in chunks of queries, band re-scoring with its certificate,
// and the exact SIMT scan for the queries that fail it.
int tc_build_knn(const RowDesc &X, int64_t n, int K, uint8_t *scratch, size_t bytes, uint64_t *keys,
                 int64_t *out_fallback, cudaStream_t st) {
    const int d = X.d, kp = (d + KA - 1) / KA * KA;
    const TcBuildLayout L = tc_build_layout(n, d, K);
    if (bytes < L.total) return fail(SVF_EINVAL, "build scratch of %zu bytes, need %zu", bytes, L.total);
    const bool u8 = X.dtype == SVF_U8;
    const float *Xf = reinterpret_cast<const float *>(X.base);
    const uint8_t *X8 = X.base;
    auto *xb = reinterpret_cast<__nv_bfloat16 *>(scratch + L.xb);
    float *norms = reinterpret_cast<float *>(scratch + L.norms);
    unsigned int *maxn = reinterpret_cast<unsigned int *>(scratch + L.maxn);
    float *cd = reinterpret_cast<float *>(scratch + L.cd);
    uint32_t *ci = reinterpret_cast<uint32_t *>(scratch + L.ci);
    int32_t *flagged = reinterpret_cast<int32_t *>(scratch + L.flagged);
    unsigned long long *nflag = reinterpret_cast<unsigned long long *>(scratch + L.nflag);
    unsigned long long *status = nflag + 8;
    if (u8)
        u8_to_bf16_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(X8, n, d, kp, xb, norms);
    else
        to_bf16_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(Xf, n, d, kp, xb, norms);
    CUDA_TRY(cudaMemsetAsync(maxn, 0, 4, st));
    CUDA_TRY(cudaMemsetAsync(status, 0, 8, st));
    max_kernel<<<296, 256, 0, st>>>(norms, n, maxn);
    const int splits = build_splits(K);
    const int wpb = 4;
    const size_t bsm = (size_t)wpb * KP * 4;
    // Rows whose certificate failed wait in gself (absolute ids) until a
    // chunk's worth has gathered; the exact SIMT scan then handles them in one
    // launch (its grid is one block per 32 queries, so a few hundred rows per
    // chunk would leave most SMs idle while every block reads the whole store).
    float *gq = reinterpret_cast<float *>(scratch + L.gq);
    uint64_t *gk = reinterpret_cast<uint64_t *>(scratch + L.gk);
    int64_t *gself = reinterpret_cast<int64_t *>(scratch + L.gself);
    int64_t fallback = 0, npend = 0;
    // band re-scoring of nq queries (rows q0.., or rows qids[..]) from `lists`
    // candidate lists into kq[nq][K]; failing queries (local indices) land in
    // flagged / nflag
    const float eps_c = u8 ? 0.f : kBf16ErrC;  // uint8: the approximate distances are exact
    auto band = [&](int lists, int64_t q0, int64_t nq, uint64_t *kq, const int64_t *qids) {
        const dim3 g((unsigned)((nq + wpb - 1) / wpb)), b(wpb * 32);
        if (lists * KC <= 32 * 8) {
            if (u8)
                band_rescore_kernel<8, true><<<g, b, bsm, st>>>(X8, d, X.metric, maxn, lists, cd, ci, q0, nq, K, eps_c,
                                                                 kq, flagged, nflag, qids);
            else
                band_rescore_kernel<8, false><<<g, b, bsm, st>>>(Xf, d, X.metric, maxn, lists, cd, ci, q0, nq, K, eps_c,
                                                                  kq, flagged, nflag, qids);
        } else {
            if (u8)
                band_rescore_kernel<16, true><<<g, b, bsm, st>>>(X8, d, X.metric, maxn, lists, cd, ci, q0, nq, K, eps_c,
                                                                  kq, flagged, nflag, qids);
            else
                band_rescore_kernel<16, false><<<g, b, bsm, st>>>(Xf, d, X.metric, maxn, lists, cd, ci, q0, nq, K,
                                                                   eps_c, kq, flagged, nflag, qids);
        }
        return cudaGetLastError();
    };
    auto flush = [&]() -> int {
        if (npend == 0) return SVF_OK;
        if (u8)
            gather_ids_u8_kernel<<<(unsigned)((npend * d + 255) / 256), 256, 0, st>>>(
                X8, d, gself, npend, reinterpret_cast<uint8_t *>(gq));
        else
            gather_ids_kernel<<<(unsigned)((npend * d + 255) / 256), 256, 0, st>>>(Xf, d, gself, npend, gq);
        KnnArgs ka{};
        ka.X = X;
        ka.n = n;
        ka.Q = gq;
        ka.q_row_bytes = u8 ? d : d * 4;
        ka.nq = npend;
        ka.self = gself;
        ka.self_base = -1;
        ka.k = K;
        ka.out_keys = gk;
        // the candidate lists are free here: a small batch is scanned in slices
        ka.part_keys = reinterpret_cast<uint64_t *>(cd);
        ka.part_bytes = (size_t)L.chunk * (2 * splits) * KC * sizeof(float);
        CUDA_TRY(launch_knn(ka, st));
        scatter_ids_kernel<<<(unsigned)((npend * K + 255) / 256), 256, 0, st>>>(gk, gself, npend, K, keys);
        CUDA_TRY(cudaGetLastError());
        fallback += npend;
        npend = 0;
        return SVF_OK;
    };
    // The pending rows first get a second pass of the same scan with twice
    // the slices (each list covers half the rows, so its 16th entry -- the
    // certificate's bound -- lies further out and the band has more
    // candidates), in batches that fit the candidate buffers; the rows it
    // certifies skip the SIMT scan.  Skipped when twice the lists exceed the
    // re-score's 512 candidates (2R = 128).
    const int splits2 = 2 * splits, lists2 = 2 * splits2;
    auto resolve = [&]() -> int {
        if (npend > 0 && lists2 * KC <= 32 * kBuildNPLMax) {
            int64_t *gfail = reinterpret_cast<int64_t *>(scratch + L.gfail);
            auto *qb2 = reinterpret_cast<__nv_bfloat16 *>(gq);  // m x kp bf16 fits the fp32 query rows' space
            const int64_t B2 = L.chunk / 2;
            int64_t nfail = 0;
            for (int64_t p0 = 0; p0 < npend; p0 += B2) {
                const int64_t m = std::min(B2, npend - p0);
                gather_bf16_kernel<<<(unsigned)((m * kp + 255) / 256), 256, 0, st>>>(xb, kp, gself + p0, m, qb2);
                TcPass p2{};
                p2.xb = xb;
                p2.qb = qb2;
                p2.n = n;
                p2.nq = m;
                p2.kp = kp;
                p2.metric = X.metric;
                p2.norms = norms;
                p2.cd = cd;
                p2.ci = ci;
                p2.seed = reinterpret_cast<float *>(scratch + L.seed);
                p2.status = status;
                if (int rc = tc_pass(p2, splits2, splits2, st)) return rc;
                CUDA_TRY(cudaMemsetAsync(nflag, 0, 8, st));
                CUDA_TRY(band(lists2, 0, m, gk, gself + p0));
                // every row's keys to its place (a failed row's pads are overwritten by the SIMT scan)
                scatter_ids_kernel<<<(unsigned)((m * K + 255) / 256), 256, 0, st>>>(gk, gself + p0, m, K, keys);
                CUDA_TRY(cudaGetLastError());
                unsigned long long hf[2] = {0, 0};
                CUDA_TRY(cudaMemcpyAsync(&hf[0], nflag, 8, cudaMemcpyDeviceToHost, st));
                CUDA_TRY(cudaMemcpyAsync(&hf[1], status, 8, cudaMemcpyDeviceToHost, st));
                CUDA_TRY(cudaStreamSynchronize(st));
                if (hf[1]) return fail(SVF_ETIMEOUT, "build: a tensor-core pipeline wait gave up");
                const int64_t mf = (int64_t)hf[0];
                if (mf > 0) {
                    pick_ids_kernel<<<(unsigned)((mf + 255) / 256), 256, 0, st>>>(flagged, mf, gself + p0, gfail + nfail);
                    CUDA_TRY(cudaGetLastError());
                }
                nfail += mf;
            }
            if (nfail > 0) CUDA_TRY(cudaMemcpyAsync(gself, gfail, (size_t)nfail * 8, cudaMemcpyDeviceToDevice, st));
            npend = nfail;
        }
        return flush();
    };
    for (int64_t q0 = 0; q0 < n; q0 += L.chunk) {
        const int64_t nq = std::min(L.chunk, n - q0);
        TcPass pass{};
        pass.xb = xb;
        pass.qb = xb + q0 * kp;  // the queries are rows of the store (16-byte aligned: kp is a multiple of 32)
        pass.n = n;
        pass.nq = nq;
        pass.kp = kp;
        pass.metric = X.metric;
        pass.norms = norms;
        pass.cd = cd;
        pass.ci = ci;
        pass.seed = reinterpret_cast<float *>(scratch + L.seed);
        pass.status = status;
        if (int rc = tc_pass(pass, splits, splits, st)) return rc;
        CUDA_TRY(cudaMemsetAsync(nflag, 0, 8, st));
        CUDA_TRY(band(2 * splits, q0, nq, keys + q0 * K, nullptr));
        unsigned long long hf[2] = {0, 0};
        CUDA_TRY(cudaMemcpyAsync(&hf[0], nflag, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(&hf[1], status, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (hf[1]) return fail(SVF_ETIMEOUT, "build: a tensor-core pipeline wait gave up");
        const int64_t m = (int64_t)hf[0];
        if (m > 0) {
            if (npend + m > L.chunk)
                if (int rc = resolve()) return rc;
            self_ids_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(flagged, m, q0, gself + npend);
            CUDA_TRY(cudaGetLastError());
            npend += m;
        }
    }
    if (int rc = resolve()) return rc;
    if (out_fallback) *out_fallback = fallback;
    return SVF_OK;
}

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
    const int kp = (d + KA - 1) / KA * KA;
    to_bf16_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(X, n, d, kp, xb, norms);
    to_bf16_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, st>>>(Q, nq, d, kp, qb, nullptr);
    CUDA_TRY(cudaMemsetAsync(maxn, 0, 4, st));
    CUDA_TRY(cudaMemsetAsync(nflag, 0, 8, st));
    max_kernel<<<296, 256, 0, st>>>(norms, n, maxn);
    // the status word of a stand-alone call lives in the flag counter's slot
    unsigned long long *status = nflag + 8;
    CUDA_TRY(cudaMemsetAsync(status, 0, 8, st));
    TcPass pass{};
    pass.xb = xb;
    pass.qb = qb;
    pass.n = n;
    pass.nq = nq;
    pass.kp = kp;
    pass.metric = metric;
    pass.norms = norms;
    pass.cd = cd;
    pass.ci = ci;
    pass.seed = reinterpret_cast<float *>(S + L.seed);
    pass.status = status;
    if (int rc = tc_pass(pass, 1, 64, st)) return rc;
    TcArgs a{};
    a.splits = pass.splits;
    const int wpb = 4;
    const size_t rsm = (size_t)wpb * a.splits * HALVES * KC * 8;
    CUDA_TRY(cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    rescore_kernel<<<(unsigned)((nq + wpb - 1) / wpb), wpb * 32, rsm, st>>>(X, Q, d, metric, norms, maxn, a.splits * HALVES, cd,
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
