// svf_dev.cuh -- device building blocks of the SVFusion graph-ANNS hot path
// for B300 (sm_103a): (distance, id) keys, the counter-based generator of the
// random pool initialisation (Alg. 1), warp-wide bitonic sort/merge of keys,
// and team-of-8-lanes distance evaluation over 16-byte row chunks.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "../../include/svf.h"

namespace svf {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr uint32_t kIdMask = 0x3FFFFFFFu;          // ids < 2^30
constexpr uint32_t kExpBit = 0x80000000u;          // pool entry already expanded
constexpr uint32_t kNewBit = 0x40000000u;          // admitted in this iteration
constexpr uint64_t kCmpMask = 0xFFFFFFFF3FFFFFFFull;  // order ignores both flags
constexpr uint64_t kPad = 0xFFFFFFFFFFFFFFFFull;   // +inf, flags set, id EMPTY
constexpr int kTeam = 8;                           // lanes per distance
constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------- keys
// A 64-bit key is (distance key << 32) | id, compared with the flag bits
// masked, so keys order lexicographically by (distance, id).
__device__ __forceinline__ uint64_t cmpk(uint64_t k) { return k & kCmpMask; }

// Order-preserving map of a float to uint32 (-0 folded into +0).
__device__ __forceinline__ uint32_t fkey(float f) {
    if (f == 0.0f) f = 0.0f;
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}
__device__ __forceinline__ uint64_t make_key(uint32_t dk, uint32_t id) {
    return ((uint64_t)dk << 32) | id;
}
__device__ __forceinline__ uint32_t key_id(uint64_t k) { return (uint32_t)k & kIdMask; }
__device__ __forceinline__ bool key_is_pad(uint64_t k) { return (uint32_t)(k >> 32) == 0xFFFFFFFFu; }

// ---------------------------------------------------------------- generator
// splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): one counter-based mixing step.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool is_deleted(const uint32_t *__restrict__ del, uint32_t id) {
    return (__ldg(del + (id >> 5)) >> (id & 31)) & 1u;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src), hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl64_xor(uint64_t v, int m) {
    uint32_t lo = __shfl_xor_sync(kFull, (uint32_t)v, m), hi = __shfl_xor_sync(kFull, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ void cswap_keep(uint64_t &a, uint64_t other, bool keep_min) {
    bool less = cmpk(other) < cmpk(a);
    if (less == keep_min) a = other;
}

// ---------------------------------------------------------------- warp sorts
// N = 32*S keys in a warp: element e = s*32 + lane lives in k[s] of `lane`.
// Full bitonic sort, ascending.
template <int S>
__device__ __forceinline__ void warp_sort(uint64_t (&k)[S], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * S; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int ss = stride >> 5;
#pragma unroll
                for (int s = 0; s < S; s++) {
                    if (s & ss) continue;
                    const int e = s * 32 + lane;
                    const bool asc = (e & size) == 0;
                    uint64_t a = k[s], b = k[s | ss];
                    bool sw = (cmpk(b) < cmpk(a)) == asc;
                    k[s] = sw ? b : a;
                    k[s | ss] = sw ? a : b;
                }
            } else {
#pragma unroll
                for (int s = 0; s < S; s++) {
                    const int e = s * 32 + lane;
                    const bool asc = (e & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    uint64_t o = shfl64_xor(k[s], stride);
                    cswap_keep(k[s], o, lower == asc);
                }
            }
        }
    }
}

// Sort a bitonic sequence of 32*S keys ascending (half-cleaner cascade).
template <int S>
__device__ __forceinline__ void warp_bitonic_merge(uint64_t (&k)[S], int lane) {
#pragma unroll
    for (int stride = 16 * S; stride > 0; stride >>= 1) {
        if (stride >= 32) {
            const int ss = stride >> 5;
#pragma unroll
            for (int s = 0; s < S; s++) {
                if (s & ss) continue;
                uint64_t a = k[s], b = k[s | ss];
                bool sw = cmpk(b) < cmpk(a);
                k[s] = sw ? b : a;
                k[s | ss] = sw ? a : b;
            }
        } else {
#pragma unroll
            for (int s = 0; s < S; s++) {
                uint64_t o = shfl64_xor(k[s], stride);
                cswap_keep(k[s], o, (lane & stride) == 0);
            }
        }
    }
}

// pool (32*LW, sorted) <- the 32*LW smallest of pool and cand (32*S, sorted).
template <int LW, int S>
__device__ __forceinline__ void warp_merge_into(uint64_t (&pool)[LW], const uint64_t (&cand)[S], int lane) {
    static_assert(S <= LW, "candidate list longer than the pool");
#pragma unroll
    for (int s = LW - S; s < LW; s++) {
        uint64_t r = shfl64(cand[LW - 1 - s], 31 - lane);
        if (cmpk(r) < cmpk(pool[s])) pool[s] = r;
    }
    warp_bitonic_merge<LW>(pool, lane);
}

// pool (32*LW, sorted) <- the 32*LW smallest of pool and {c}: c's rank is
// counted by ballots, entries from that rank on move up one place (the
// last one leaves) and c takes the freed slot.  Keys are distinct, so a
// sequence of these gives the same pool as sorting and merging the set.
template <int LW>
__device__ __forceinline__ void warp_insert_one(uint64_t (&pool)[LW], uint64_t c, int lane) {
    const uint64_t cc = cmpk(c);
    int r = 0;
#pragma unroll
    for (int s = 0; s < LW; s++) r += __popc(__ballot_sync(kFull, cmpk(pool[s]) < cc));
    if (r >= 32 * LW) return;
#pragma unroll
    for (int s = LW - 1; s >= 0; s--) {  // downwards: pool[s - 1] is still the old row here
        uint32_t lo = __shfl_up_sync(kFull, (uint32_t)pool[s], 1), hi = __shfl_up_sync(kFull, (uint32_t)(pool[s] >> 32), 1);
        uint64_t up = ((uint64_t)hi << 32) | lo;
        if (s > 0) {
            const uint64_t last = shfl64(pool[s - 1], 31);
            if (lane == 0) up = last;
        }
        const int e = s * 32 + lane;
        if (e >= r) pool[s] = e == r ? c : up;
    }
}

// pool (32*LW, sorted) <- the 32*LW smallest of pool and the real keys of
// cand (32*S keys in any order, kPad where empty, none equal to a pool key),
// every key placed at once: a pool entry moves up by the number of
// candidates below it, a candidate lands at (pool entries below it) +
// (candidates below it).  The keys are scattered through `buf` (32*LW keys of
// shared memory the call may overwrite).  Each candidate costs one broadcast
// and LW ballots, so this is for a few of them; the result equals inserting
// them one by one, or sorting and merging the set.
template <int LW, int S>
__device__ __forceinline__ void warp_insert_few(uint64_t (&pool)[LW], const uint64_t (&cand)[S], uint64_t *buf,
                                                int lane) {
    constexpr int L = 32 * LW;
    uint64_t cp[LW], cc[S];
    uint32_t below[LW];  // candidates below each pool entry
    int pos[S];          // final place of each candidate
#pragma unroll
    for (int s = 0; s < LW; s++) {
        cp[s] = cmpk(pool[s]);
        below[s] = 0;
    }
#pragma unroll
    for (int s = 0; s < S; s++) {
        cc[s] = cmpk(cand[s]);
        pos[s] = 0;
    }
#pragma unroll
    for (int cs = 0; cs < S; cs++) {
        uint32_t m = __ballot_sync(kFull, !key_is_pad(cand[cs]));
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            const uint64_t c = shfl64(cc[cs], src);
            int r = 0;
#pragma unroll
            for (int s = 0; s < LW; s++) {
                below[s] += c < cp[s];
                r += __popc(__ballot_sync(kFull, cp[s] < c));
            }
#pragma unroll
            for (int s = 0; s < S; s++) pos[s] += c < cc[s];
            if (lane == src) pos[cs] += r;
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < LW; s++) {
        const int p = s * 32 + lane + (int)below[s];
        if (p < L) buf[p] = pool[s];
    }
#pragma unroll
    for (int s = 0; s < S; s++)
        if (!key_is_pad(cand[s]) && pos[s] < L) buf[pos[s]] = cand[s];
    __syncwarp();
#pragma unroll
    for (int s = 0; s < LW; s++) pool[s] = buf[s * 32 + lane];
    __syncwarp();
}

// ---------------------------------------------------------------- distances
// A row is split into 16-byte chunks; the 8 lanes of a team take chunks
// sub, sub+8, sub+16, ... and the partial sums are combined by xor shuffles
// within the team, in a fixed order.  The query sits in shared memory as
// fp32 (uint8 for a U8 index) in the same chunk layout as the row's values.
struct RowDesc {
    const uint8_t *base;  // store base
    int64_t pitch;        // bytes per row
    int nchunk;           // 16-byte chunks of values per row
    int d;
    int dtype;            // traversal dtype
    int metric;
    int copy_bytes;       // bytes staged per row (values, + the FP8 scale), multiple of 16
    int ts;               // lanes per row when staged (power of two, <= 32)
    int cpl;              // chunks per lane = ceil(nchunk / ts)
    const int32_t *map;   // tiered store: device cache slot of each id (-1: host row), or null
    const uint8_t *host;  // tiered store: all rows in mapped pinned host memory
};

// Address of row `id`: the store itself, or for a tiered store its device
// cache slot when cached and its host row otherwise (host memory is read
// through the mapping; the tier tables do not change while a kernel runs).
__device__ __forceinline__ const uint8_t *row_ptr(const RowDesc &R, uint32_t id) {
    if (R.map) {
        const int32_t s = __ldg(R.map + id);
        return s >= 0 ? R.base + (int64_t)s * R.pitch : R.host + (int64_t)id * R.pitch;
    }
    return R.base + (int64_t)id * R.pitch;
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}
__device__ __forceinline__ float l2_4(float4 q, float4 x, float acc) {
    float dx = q.x - x.x, dy = q.y - x.y, dz = q.z - x.z, dw = q.w - x.w;
    acc = fmaf(dx, dx, acc);
    acc = fmaf(dy, dy, acc);
    acc = fmaf(dz, dz, acc);
    return fmaf(dw, dw, acc);
}
__device__ __forceinline__ float4 bf2_to_f4(uint32_t a, uint32_t b) {
    return make_float4(__uint_as_float(a << 16), __uint_as_float(a & 0xFFFF0000u), __uint_as_float(b << 16),
                       __uint_as_float(b & 0xFFFF0000u));
}
// Packed fp32 pairs (Blackwell f32x2 instructions): each half is an
// independent IEEE fp32 lane, rounded as the scalar instruction would be.
__device__ __forceinline__ uint64_t f2pack(float lo, float hi) {
    return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float f2sum(uint64_t p) {
    return __uint_as_float((uint32_t)p) + __uint_as_float((uint32_t)(p >> 32));
}
// a.xy . b.xy + a.zw . b.zw into the two packed accumulators (IP), or
// (a - s b)^2 summed likewise (L2; s = 1 for bf16)
__device__ __forceinline__ void dot4_2(float4 q, float2 x01, float2 x23, uint64_t (&p)[2]) {
    p[0] = ffma2(f2pack(q.x, q.y), f2pack(x01.x, x01.y), p[0]);
    p[1] = ffma2(f2pack(q.z, q.w), f2pack(x23.x, x23.y), p[1]);
}
__device__ __forceinline__ void l2_4_2(float4 q, float2 x01, float2 x23, uint64_t nscale2, uint64_t (&p)[2]) {
    const uint64_t d0 = ffma2(f2pack(x01.x, x01.y), nscale2, f2pack(q.x, q.y));  // q - s x, one rounding
    const uint64_t d1 = ffma2(f2pack(x23.x, x23.y), nscale2, f2pack(q.z, q.w));
    p[0] = ffma2(d0, d0, p[0]);
    p[1] = ffma2(d1, d1, p[1]);
}
__device__ __forceinline__ float2 fp8x2_to_f2(uint32_t w16) {
    __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w16 & 0xFFFFu), __NV_E4M3);
    return __half22float2(*reinterpret_cast<__half2 *>(&h));
}

__device__ __forceinline__ float4 fp8x4_to_f4(uint32_t w) {
    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    float2 a = __half22float2(*reinterpret_cast<__half2 *>(&lo));
    float2 b = __half22float2(*reinterpret_cast<__half2 *>(&hi));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Partial (per-lane) accumulation of one 16-byte row chunk `c` against the
// query.  qf: fp32 query in smem; qb: uint8 query in smem.  For FP8 the
// values are codes; IP multiplies by the scale after the reduction, L2
// applies it per element.
template <int DT>
__device__ __forceinline__ void chunk_acc(int metric, const uint4 v, int c, const float *qf, const uint8_t *qb,
                                          float scale, float &facc, uint32_t &iacc, uint64_t (&pacc)[2]) {
    if constexpr (DT == SVF_F32) {
        float4 x = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                               __uint_as_float(v.w));
        float4 q = reinterpret_cast<const float4 *>(qf)[c];
        facc = metric == SVF_L2 ? l2_4(q, x, facc) : dot4(q, x, facc);
    } else if constexpr (DT == SVF_U8) {
        uint4 q = reinterpret_cast<const uint4 *>(qb)[c];
        if (metric == SVF_L2) {
            uint32_t a = __vabsdiffu4(v.x, q.x), b = __vabsdiffu4(v.y, q.y), e = __vabsdiffu4(v.z, q.z),
                     f = __vabsdiffu4(v.w, q.w);
            iacc = __dp4a(a, a, iacc);
            iacc = __dp4a(b, b, iacc);
            iacc = __dp4a(e, e, iacc);
            iacc = __dp4a(f, f, iacc);
        } else {
            iacc = __dp4a(v.x, q.x, iacc);
            iacc = __dp4a(v.y, q.y, iacc);
            iacc = __dp4a(v.z, q.z, iacc);
            iacc = __dp4a(v.w, q.w, iacc);
        }
    } else if constexpr (DT == SVF_BF16) {
        // packed pairs, two accumulators (four fp32 partial sums per lane)
        const float4 *q = reinterpret_cast<const float4 *>(qf) + 2 * c;
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        const uint64_t m1 = f2pack(-1.f, -1.f);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float2 x01 = make_float2(__uint_as_float(w[2 * h] << 16), __uint_as_float(w[2 * h] & 0xFFFF0000u));
            const float2 x23 =
                make_float2(__uint_as_float(w[2 * h + 1] << 16), __uint_as_float(w[2 * h + 1] & 0xFFFF0000u));
            if (metric == SVF_L2)
                l2_4_2(q[h], x01, x23, m1, pacc);
            else
                dot4_2(q[h], x01, x23, pacc);
        }
    } else {  // FP8: codes; IP scales after the sum, L2 scales each code
        const float4 *q = reinterpret_cast<const float4 *>(qf) + 4 * c;
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        const uint64_t ns2 = f2pack(-scale, -scale);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float2 x01 = fp8x2_to_f2(w[u]), x23 = fp8x2_to_f2(w[u] >> 16);
            if (metric == SVF_L2)
                l2_4_2(q[u], x01, x23, ns2, pacc);
            else
                dot4_2(q[u], x01, x23, pacc);
        }
    }
}

// fold the packed partial sums of a low-precision row into facc
template <int DT>
__device__ __forceinline__ void fold_pacc(float &facc, const uint64_t (&pacc)[2]) {
    if constexpr (DT == SVF_BF16 || DT == SVF_FP8) facc = f2sum(pacc[0]) + f2sum(pacc[1]);
}

template <int DT>
__device__ __forceinline__ uint32_t finish_key(int metric, float facc, uint32_t iacc, float scale) {
    if constexpr (DT == SVF_U8) {
        // L2: the exact non-negative int; IP: -dot through the order-
        // preserving int32 -> uint32 map (sign bit flipped).
        if (metric == SVF_L2) return iacc;
        return (uint32_t)(-(int32_t)iacc) ^ 0x80000000u;
    } else {
        if (DT == SVF_FP8 && metric == SVF_IP) facc *= scale;
        return fkey(metric == SVF_L2 ? facc : -facc);
    }
}

// Distance keys of two rows for one team of 8 lanes (valid flags are
// uniform within the team).  Every chunk load of both rows is issued before
// any arithmetic so a team keeps up to 2 x 4 x 16 B per lane in flight.
template <int DT>
__device__ __forceinline__ void team_dist_key2(const RowDesc &R, uint32_t ida, bool va, uint32_t idb, bool vb,
                                               int sub, const float *qf, const uint8_t *qb, uint32_t &ka,
                                               uint32_t &kb) {
    float fa = 0.0f, fb = 0.0f, sa = 1.0f, sb = 1.0f;
    uint32_t ia = 0, ib = 0;
    uint64_t pa[2] = {0, 0}, pb[2] = {0, 0};
    const uint8_t *ra = row_ptr(R, ida);
    const uint8_t *rb = row_ptr(R, idb);
    if (DT == SVF_FP8) {
        if (va) sa = __ldg(reinterpret_cast<const float *>(ra + R.d));
        if (vb) sb = __ldg(reinterpret_cast<const float *>(rb + R.d));
    }
    for (int c0 = sub; c0 < R.nchunk; c0 += 4 * kTeam) {
        uint4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int c = c0 + u * kTeam;
            if (va && c < R.nchunk) a[u] = __ldg(reinterpret_cast<const uint4 *>(ra) + c);
            if (vb && c < R.nchunk) b[u] = __ldg(reinterpret_cast<const uint4 *>(rb) + c);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int c = c0 + u * kTeam;
            if (va && c < R.nchunk) chunk_acc<DT>(R.metric, a[u], c, qf, qb, sa, fa, ia, pa);
            if (vb && c < R.nchunk) chunk_acc<DT>(R.metric, b[u], c, qf, qb, sb, fb, ib, pb);
        }
    }
    fold_pacc<DT>(fa, pa);
    fold_pacc<DT>(fb, pb);
#pragma unroll
    for (int m = kTeam / 2; m > 0; m >>= 1) {
        if constexpr (DT == SVF_U8) {
            ia += __shfl_xor_sync(kFull, ia, m);
            ib += __shfl_xor_sync(kFull, ib, m);
        } else {
            fa += __shfl_xor_sync(kFull, fa, m);
            fb += __shfl_xor_sync(kFull, fb, m);
        }
    }
    ka = finish_key<DT>(R.metric, fa, ia, sa);
    kb = finish_key<DT>(R.metric, fb, ib, sb);
}

// Keys of list[0..n) written to keys[0..n) (id | flags): 8 rows per warp step.
template <int DT>
__device__ __forceinline__ void dist_list(const RowDesc &R, const uint32_t *list, int n, uint64_t *keys,
                                          uint32_t flags, int lane, const float *qf, const uint8_t *qb) {
    const int team = lane >> 3, sub = lane & 7;
    for (int i0 = 0; i0 < n; i0 += 2 * (32 / kTeam)) {
        int ia = i0 + team, ib = i0 + (32 / kTeam) + team;
        bool va = ia < n, vb = ib < n;
        uint32_t ida = va ? list[ia] : 0u, idb = vb ? list[ib] : 0u;
        uint32_t ka, kb;
        team_dist_key2<DT>(R, ida, va, idb, vb, sub, qf, qb, ka, kb);
        if (sub == 0) {
            if (va) keys[ia] = make_key(ka, ida | flags);
            if (vb) keys[ib] = make_key(kb, idb | flags);
        }
    }
}

// Distance key between two rows of a primary store (F32 or U8), one team:
// lane `sub` takes chunks sub, sub+8, ...; the same chunk order and
// arithmetic as the query path, so dist(x_u, x_v) computed here equals the
// search kernel's dist(q = x_v, x_u) bit for bit.
template <int DT>
__device__ __forceinline__ uint32_t team_pair_key(int metric, const uint4 *ra, const uint4 *rb, int nchunk, int sub) {
    float f = 0.0f;
    uint32_t ia = 0;
    for (int c0 = sub; c0 < nchunk; c0 += 4 * kTeam) {
        uint4 va[4], vb[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int c = c0 + u * kTeam;
            if (c < nchunk) {
                va[u] = ra[c];
                vb[u] = rb[c];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            int c = c0 + u * kTeam;
            if (c >= nchunk) continue;
            if constexpr (DT == SVF_U8) {
                if (metric == SVF_L2) {
                    uint32_t a = __vabsdiffu4(vb[u].x, va[u].x), b = __vabsdiffu4(vb[u].y, va[u].y),
                             e = __vabsdiffu4(vb[u].z, va[u].z), g = __vabsdiffu4(vb[u].w, va[u].w);
                    ia = __dp4a(a, a, ia);
                    ia = __dp4a(b, b, ia);
                    ia = __dp4a(e, e, ia);
                    ia = __dp4a(g, g, ia);
                } else {
                    ia = __dp4a(vb[u].x, va[u].x, ia);
                    ia = __dp4a(vb[u].y, va[u].y, ia);
                    ia = __dp4a(vb[u].z, va[u].z, ia);
                    ia = __dp4a(vb[u].w, va[u].w, ia);
                }
            } else {
                float4 qa = make_float4(__uint_as_float(va[u].x), __uint_as_float(va[u].y), __uint_as_float(va[u].z),
                                        __uint_as_float(va[u].w));
                float4 xb = make_float4(__uint_as_float(vb[u].x), __uint_as_float(vb[u].y), __uint_as_float(vb[u].z),
                                        __uint_as_float(vb[u].w));
                f = metric == SVF_L2 ? l2_4(qa, xb, f) : dot4(qa, xb, f);
            }
        }
    }
#pragma unroll
    for (int m = kTeam / 2; m > 0; m >>= 1) {
        if constexpr (DT == SVF_U8)
            ia += __shfl_xor_sync(kFull, ia, m, kTeam);
        else
            f += __shfl_xor_sync(kFull, f, m, kTeam);
    }
    return finish_key<DT>(metric, f, ia, 1.0f);
}

// ---------------------------------------------------------------- versions
// Searches that overlap updates (the serving loop's update stream, Sec. 4.4,
// with the consistency of Sec. 5.3).  Update number E (1, 2, ...) stamps
// every existing graph row it rewrites with row_ver = E, after copying the
// row's previous content into a shadow row, and every vertex it deletes with
// del_ep = E before setting its bit.  A search of epoch e (the updates it
// must see) reads a row stamped later than e from its shadow and treats a
// vertex deleted later than e as live; vertices inserted later than e have
// ids >= its n_used and are never named.  One shadow per row suffices: the
// serving loop starts update E + 1 only after every search of an epoch
// below E has finished.
struct VerCtx {
    const uint32_t *row_ver;     // [n_cap] update that last rewrote the row (0: none), or null: no versions
    const int32_t *shadow_slot;  // [n_cap] shadow row holding the content before that update
    const uint32_t *shadow;      // [slots][R]
    const uint32_t *del_ep;      // [n_cap] update that deleted the vertex (where its bit is set)
    uint32_t epoch;              // the search's epoch
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Graph row p (R = 32 S entries; lane l gets entries l, l + 32, ...) as a
// search of epoch v.epoch sees it.  A row rewritten during the read is
// detected by reading its stamp again after the row (the update stamps a row
// before any kernel writes it), and is then read from its shadow.
template <int S>
__device__ __forceinline__ void versioned_row(const VerCtx &v, const uint32_t *graph, uint32_t p, int lane,
                                              uint32_t (&nb)[S]) {
    constexpr int R = 32 * S;
    uint32_t ver = ld_acquire_u32(v.row_ver + p);
    if (ver <= v.epoch) {
#pragma unroll
        for (int s = 0; s < S; s++) nb[s] = __ldcg(graph + (int64_t)p * R + s * 32 + lane);
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        ver = ld_acquire_u32(v.row_ver + p);
        if (ver <= v.epoch) return;
    }
    const int32_t slot = (int32_t)ld_relaxed_u32(reinterpret_cast<const uint32_t *>(v.shadow_slot) + p);
#pragma unroll
    for (int s = 0; s < S; s++) nb[s] = __ldcg(v.shadow + (int64_t)slot * R + s * 32 + lane);
}

// Deleted as of the search's epoch: its bit is set and its deletion was not
// later than the epoch (a concurrent deletion is later: its del_ep is either
// still unset, 0xFFFFFFFF, or already its own number, both above the epoch).
__device__ __forceinline__ bool deleted_at(const VerCtx &v, const uint32_t *__restrict__ del, uint32_t id) {
    if (!((__ldcg(del + (id >> 5)) >> (id & 31)) & 1u)) return false;
    return ld_relaxed_u32(v.del_ep + id) <= v.epoch;
}

// Output value of a distance key: float, or int32 for a U8 store.
__device__ __forceinline__ uint32_t key_to_out(uint32_t dk, int dtype, int metric) {
    if (dk == 0xFFFFFFFFu) return dtype == SVF_U8 ? 0x7FFFFFFFu : 0x7F800000u;  // INT32_MAX / +inf
    if (dtype == SVF_U8) return metric == SVF_L2 ? dk : (dk ^ 0x80000000u);
    return __float_as_uint(fkey_inv(dk));
}

// Status block layout (uint64 words).
enum StatusWord {
    kStError = 0,     // first device-side error code (int, 0 = none)
    kStDetail = 1,    // detail of that error
    kStQueries = 2,
    kStIters = 3,
    kStEvals = 4,
    kStResets = 5,
    kStRepaired = 6,
    kStRevTargets = 7,
    kStNewlyDeleted = 8,
    kStHits = 9,       // tiered store: distance rows read from the device cache
    kStMisses = 10,    // tiered store: rows read from host memory
    kStQCount = 11,    // tiered store: promotion candidates queued
    kStPromoted = 12,  // tiered store: rows promoted into the cache
    kStEvicted = 13,   // tiered store: cached rows evicted
    kStScratch0 = 16,  // per-call scratch counters
    kStWords = 64
};

__device__ __forceinline__ void set_error(unsigned long long *st, int code, long long detail) {
    if (atomicCAS(st + kStError, 0ull, (unsigned long long)(unsigned)(-code)) == 0ull)
        st[kStDetail] = (unsigned long long)detail;
}

}  // namespace svf

namespace svf {

// ---------------------------------------------------------------- staging
// Rows are brought into a per-warp shared-memory buffer by the bulk-copy
// (TMA, 1-D) engine: one cp.async.bulk per row, completion counted in bytes
// on a per-warp mbarrier.  No cluster multicast is used.
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

constexpr uint32_t kWaitLimit = 1u << 18;  // polls of an mbarrier before a wait gives up (~1 s: an idle poll suspends ~4 us)

struct Stage {
    uint8_t *buf;       // per-warp buffer (16-byte aligned)
    uint32_t cap;       // bytes
    uint64_t *mbar;     // two per-warp mbarriers: first and second half of a batch
    uint32_t phase[2];  // parity of the next phase to wait for, per barrier
};

// Workload-aware placement state used on cache misses (SVFusion Sec. 4.3):
// F_lambda(x) = alpha * F_recent(x) + beta * log(1 + E_in(x)); a missed x with
// F_lambda > theta is queued for promotion (once: bit 31 of freq marks it).
struct TierCtx {
    uint8_t *ref;          // clock reference bit per cache slot
    uint32_t *freq;        // F_recent per id (bit 31: queued)
    const uint32_t *ein;   // E_in per id
    uint32_t *queue;       // promotion candidates
    unsigned long long *qcount;
    uint32_t qcap;
    float alpha, beta, theta;
    uint32_t *stat;        // per slot, 2 words: LRU [last hit stamp, -], LRFU [hits this round, C (f32)]; or null
    uint32_t tick;         // stamp of this call's hits (LRU)
    int lru;               // 1: LRU stamps, 0: LRFU counts (when stat is set)
};
constexpr uint32_t kQueuedBit = 0x80000000u;

// A cache hit on slot s: the reference bit (clock policies) and the LRU /
// LRFU recency state.
__device__ __forceinline__ void tier_hit(const TierCtx &T, int32_t s) {
    T.ref[s] = 1;
    if (T.stat) {
        if (T.lru)
            T.stat[2 * (int64_t)s] = T.tick;
        else
            atomicAdd(T.stat + 2 * (int64_t)s, 1u);
    }
}

__device__ __forceinline__ void tier_miss(const TierCtx &T, uint32_t id) {
    const uint32_t old = atomicAdd(T.freq + id, 1u);
    if (old & kQueuedBit) return;
    const float f = T.alpha * (float)((old & ~kQueuedBit) + 1u) + T.beta * log1pf((float)__ldg(T.ein + id));
    if (f <= T.theta) return;
    const uint32_t prev = atomicOr(T.freq + id, kQueuedBit);
    if (prev & kQueuedBit) return;
    const unsigned long long pos = atomicAdd(T.qcount, 1ull);
    if (pos < T.qcap)
        T.queue[pos] = id;
    else
        atomicAnd(T.freq + id, ~kQueuedBit);  // queue full: let a later miss queue it
}

// Staged-row layout known at compile time (NCH 16-byte value chunks per
// row): the team size and chunks per lane of set_team, and the staged row
// bytes (values, plus the scale slot for FP8).
// Chunks per lane at most: 8 for FP8 rows (one lane per d = 96 or 128 row,
// no team reduction), 4 otherwise.
__host__ __device__ constexpr int max_chunks_per_lane(int dtype) { return dtype == SVF_FP8 ? 8 : 4; }
__host__ __device__ constexpr int team_for(int nch, int dtype) {
    int ts = 1;
    while (ts < 32 && (nch + ts - 1) / ts > max_chunks_per_lane(dtype)) ts <<= 1;
    return ts;
}
template <int DT, int NCH>
__host__ __device__ constexpr int staged_row_bytes() {
    return NCH * 16 + (DT == SVF_FP8 ? 16 : 0);
}

// Distance keys of rows list[0..n) (smem ids) written to keys[0..n) with
// `flags` or'ed into the id word.  Rows are staged in chunks that fit the
// buffer; each chunk is one batch of bulk copies and one barrier wait.
// Returns false if a wait gave up (the caller reports SVF_ETIMEOUT).
// NCH > 0: the row layout is NCH chunks (the caller has checked R against
// it), so loop bounds and predicates fold at compile time.
template <int DT, int NCH = 0>
__device__ __forceinline__ bool staged_dist(Stage &S, const RowDesc &R, const uint32_t *list, int n, uint64_t *keys,
                                            uint32_t flags, int lane, const float *qf, const uint8_t *qb,
                                            const TierCtx *tier = nullptr, int *hits = nullptr, int *misses = nullptr) {
    constexpr bool CT = NCH > 0;
    const int cb = CT ? staged_row_bytes<DT, NCH>() : R.copy_bytes;
    const int nch = CT ? NCH : R.nchunk;
    const int cpl = CT ? (NCH + team_for(NCH, DT) - 1) / team_for(NCH, DT) : R.cpl;
    const int per = (int)(S.cap / (uint32_t)cb);
    const int ts = CT ? team_for(NCH, DT) : R.ts, team = lane / ts, sub = lane % ts, nteam = 32 / ts;
    for (int i0 = 0; i0 < n; i0 += per) {
        const int cnt = min(per, n - i0);
        __syncwarp();
        fence_proxy_async();  // earlier reads of the buffer precede the new async writes
        // Rows [0, h) complete on barrier 0 and [h, cnt) on barrier 1 (h a
        // whole number of team rounds), so the first half's distances are
        // computed while the second half is still arriving.
        int h = cnt;
        if (!R.map) {
            const int rounds = (cnt + nteam - 1) / nteam;
            if (rounds > 1) h = min(cnt, (rounds + 1) / 2 * nteam);
            if (lane == 0) {
                mbar_expect_tx(S.mbar, (uint32_t)(h * cb));
                if (cnt > h) mbar_expect_tx(S.mbar + 1, (uint32_t)((cnt - h) * cb));
            }
            __syncwarp();
            for (int j = lane; j < cnt; j += 32)
                bulk_g2s(S.buf + (size_t)j * cb, R.base + (int64_t)list[i0 + j] * R.pitch, cb, S.mbar + (j >= h));
            uint32_t it = 0;
            while (!mbar_try_wait(S.mbar, S.phase[0]))
                if (++it > kWaitLimit) return false;
            S.phase[0] ^= 1u;
        } else {
            // tiered store: cached rows by bulk copy from the device cache,
            // missed rows read from host memory by the lane that owns them
            int nhit = 0;
            for (int j = lane; j < cnt; j += 32) nhit += __ldg(R.map + list[i0 + j]) >= 0;
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) nhit += __shfl_xor_sync(kFull, nhit, m);
            if (nhit > 0 && lane == 0) mbar_expect_tx(S.mbar, (uint32_t)(nhit * cb));
            __syncwarp();
            uint32_t mmask = 0;  // this lane's missed rows (j = lane + 32 t)
            for (int j = lane, t = 0; j < cnt; j += 32, t++) {
                const uint32_t id = list[i0 + j];
                const int32_t slot = __ldg(R.map + id);
                if (slot >= 0) {
                    bulk_g2s(S.buf + (size_t)j * cb, R.base + (int64_t)slot * R.pitch, cb, S.mbar);
                    tier_hit(*tier, slot);
                } else {
                    mmask |= 1u << t;
                    tier_miss(*tier, id);
                }
            }
            // missed rows: the whole warp copies them from host memory, every
            // 16-byte chunk of every missed row spread over the lanes
            const int cpr = cb / 16;
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                const uint32_t miss = __ballot_sync(kFull, (mmask >> (j0 >> 5)) & 1u);
                const int nm = __popc(miss);
#pragma unroll 4
                for (int e = lane; e < nm * cpr; e += 32) {
                    const int r = e / cpr, c = e - r * cpr;
                    const int j = j0 + __fns(miss, 0, r + 1);  // position of the r-th missed row
                    const uint4 *src = reinterpret_cast<const uint4 *>(R.host + (int64_t)list[i0 + j] * R.pitch);
                    reinterpret_cast<uint4 *>(S.buf + (size_t)j * cb)[c] = src[c];
                }
            }
            if (hits) *hits += nhit;
            if (misses) *misses += cnt - nhit;
            if (nhit > 0) {
                uint32_t it = 0;
                while (!mbar_try_wait(S.mbar, S.phase[0]))
                    if (++it > kWaitLimit) return false;
                S.phase[0] ^= 1u;
            }
            __syncwarp();
        }
        // FP32 / BF16 compile-time layouts with <= 3 chunks per lane (FP8 keeps
        // the half-batch split, which measured better): each lane takes two
        // rows at once (rows r and r + nteam), so every query chunk loaded
        // from shared memory serves both and the two dependency chains
        // interleave.  The pair's second row may need the second barrier.
        constexpr bool PAIR = CT && (DT == SVF_F32 || DT == SVF_BF16) && (NCH + team_for(NCH, DT) - 1) / team_for(NCH, DT) <= 3;
        if constexpr (PAIR) {
            constexpr int TS = team_for(NCH, DT), CPL = (NCH + TS - 1) / TS, NT = 32 / TS;
            bool second = cnt <= h;
            for (int r0 = 0; r0 < cnt; r0 += 2 * NT) {
                if (!second && r0 + NT >= h) {
                    uint32_t it = 0;
                    while (!mbar_try_wait(S.mbar + 1, S.phase[1]))
                        if (++it > kWaitLimit) return false;
                    S.phase[1] ^= 1u;
                    second = true;
                }
                const int ra = r0 + team, rb = r0 + NT + team;
                const bool va = ra < cnt, vb = rb < cnt;
                const uint8_t *rowa = S.buf + (size_t)(va ? ra : 0) * cb;
                const uint8_t *rowb = S.buf + (size_t)(vb ? rb : 0) * cb;
                float fa = 0.f, fb = 0.f, sa = 1.f, sb = 1.f;
                uint32_t ia = 0, ib = 0;
                uint64_t pa[2] = {0, 0}, pb[2] = {0, 0};
                if (DT == SVF_FP8) {
                    sa = *reinterpret_cast<const float *>(rowa + R.d);
                    sb = *reinterpret_cast<const float *>(rowb + R.d);
                }
                uint4 xa[CPL], xb[CPL];
#pragma unroll
                for (int u = 0; u < CPL; u++) {
                    const int c = sub + u * TS;
                    if (c < NCH) {
                        xa[u] = reinterpret_cast<const uint4 *>(rowa)[c];
                        xb[u] = reinterpret_cast<const uint4 *>(rowb)[c];
                    }
                }
#pragma unroll
                for (int u = 0; u < CPL; u++) {
                    const int c = sub + u * TS;
                    if (c < NCH) {
                        chunk_acc<DT>(R.metric, xa[u], c, qf, qb, sa, fa, ia, pa);
                        chunk_acc<DT>(R.metric, xb[u], c, qf, qb, sb, fb, ib, pb);
                    }
                }
                fold_pacc<DT>(fa, pa);
                fold_pacc<DT>(fb, pb);
#pragma unroll
                for (int m = TS >> 1; m > 0; m >>= 1) {
                    fa += __shfl_xor_sync(kFull, fa, m);
                    fb += __shfl_xor_sync(kFull, fb, m);
                }
                if (sub == 0) {
                    if (va) keys[i0 + ra] = make_key(finish_key<DT>(R.metric, fa, ia, sa), list[i0 + ra] | flags);
                    if (vb) keys[i0 + rb] = make_key(finish_key<DT>(R.metric, fb, ib, sb), list[i0 + rb] | flags);
                }
            }
        } else {
            for (int r0 = 0; r0 < cnt; r0 += nteam) {
                if (r0 == h) {  // the second half
                    uint32_t it = 0;
                    while (!mbar_try_wait(S.mbar + 1, S.phase[1]))
                        if (++it > kWaitLimit) return false;
                    S.phase[1] ^= 1u;
                }
                const int r = r0 + team;
                const bool valid = r < cnt;
                const uint8_t *row = S.buf + (size_t)(valid ? r : 0) * cb;
                float facc = 0.f, scale = 1.f;
                uint32_t iacc = 0;
                uint64_t pacc[2] = {0, 0};
                if (DT == SVF_FP8) scale = *reinterpret_cast<const float *>(row + R.d);
                constexpr int MC = max_chunks_per_lane(DT);
                uint4 v[MC];
#pragma unroll
                for (int u = 0; u < MC; u++) {
                    const int c = sub + u * ts;
                    if (valid && u < cpl && c < nch) v[u] = reinterpret_cast<const uint4 *>(row)[c];
                }
#pragma unroll
                for (int u = 0; u < MC; u++) {
                    const int c = sub + u * ts;
                    if (valid && u < cpl && c < nch)
                        chunk_acc<DT>(R.metric, v[u], c, qf, qb, scale, facc, iacc, pacc);
                }
                for (int c0 = sub + MC * ts; c0 < nch; c0 += ts)  // rows longer than MC chunks per lane
                    if (valid)
                        chunk_acc<DT>(R.metric, reinterpret_cast<const uint4 *>(row)[c0], c0, qf, qb, scale, facc, iacc,
                                      pacc);
                fold_pacc<DT>(facc, pacc);
                for (int m = ts >> 1; m > 0; m >>= 1) {
                    if constexpr (DT == SVF_U8)
                        iacc += __shfl_xor_sync(kFull, iacc, m);
                    else
                        facc += __shfl_xor_sync(kFull, facc, m);
                }
                if (valid && sub == 0)
                    keys[i0 + r] = make_key(finish_key<DT>(R.metric, facc, iacc, scale), list[i0 + r] | flags);
            }
        }
    }
    __syncwarp();
    return true;
}

}  // namespace svf
