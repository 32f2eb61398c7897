// search_kernel.cuh -- batched greedy beam search over the fixed out-degree graph
// (SVFusion Alg. 1, Sec. 4.2), one warp per query, for sm_103a.
//
// Per warp: the query and a visited table live in shared memory; the
// candidate pool (L keys, sorted by (distance, id)) lives in registers,
// L/32 keys per lane.  Each iteration picks the nearest unexpanded pool
// entry (ballots), loads its R-entry graph row with one coalesced load,
// drops empty / deleted / visited ids (bitset + shared-memory hash insert),
// evaluates the survivors with teams of 8 lanes (128-bit row loads, shuffle
// reduction), bitonic-sorts them and merges them into the pool.
//
// Visited table: exact open addressing while it has room; when it is half
// full it is cleared and re-seeded with the current pool.  Forgetting an id
// that left the pool cannot change the result: the pool's L-th key never
// rises, so a re-evaluated id that was once rejected is rejected again.
#pragma once
#include <cstdint>

#include "svf_dev.cuh"
#include "svf_internal.h"

#ifndef SVF_SEARCH_MINB
#define SVF_SEARCH_MINB 6  // resident CTAs of 4 warps per SM the register budget aims for
#endif
#include "svf_mlp.h"

namespace svf {

// Stop-network inference (16 -> 64 relu -> 1) reads the packed bf16 layout
// of mlp.cu: W1 [64][16], b1 [64], w2 [64], b2.

// Up to this many admitted candidates are placed into the pool directly
// (ranks by ballots, scattered through shared memory); more are sorted and
// merged.  The multi-warp kernel inserts up to this many one at a time.
constexpr int kFastInsert = 8;

__device__ __forceinline__ uint32_t hash_slot(uint32_t id, int bits) { return (id * 0x9E3779B1u) >> (32 - bits); }

// Insert id; true if it was not present.  The table is kept at most half
// full, so the probe always ends; the bound is only a guard.  A plain read
// comes first: a slot that already holds a value needs no atomic (values are
// only ever written into empty slots until the table is reset).
__device__ __forceinline__ bool ht_insert(uint32_t *ht, int bits, uint32_t id) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h = hash_slot(id, bits);
    for (uint32_t p = 0; p <= mask; p++) {
        const uint32_t cur = *reinterpret_cast<volatile uint32_t *>(ht + h);
        if (cur == id) return false;
        if (cur == kEmpty) {
            const uint32_t old = atomicCAS(ht + h, kEmpty, id);
            if (old == kEmpty) return true;
            if (old == id) return false;
        }
        h = (h + 1) & mask;
    }
    return false;
}
__device__ __forceinline__ bool ht_contains(const uint32_t *ht, int bits, uint32_t id) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h = hash_slot(id, bits);
    for (uint32_t p = 0; p <= mask; p++) {
        uint32_t v = ht[h];
        if (v == id) return true;
        if (v == kEmpty) return false;
        h = (h + 1) & mask;
    }
    return false;
}

template <int LW>
__device__ __forceinline__ void ht_reset(uint32_t *ht, int bits, const uint64_t (&pool)[LW], int lane) {
    for (int i = lane; i < (1 << bits); i += 32) ht[i] = kEmpty;
    __syncwarp();
#pragma unroll
    for (int s = 0; s < LW; s++)
        if (!key_is_pad(pool[s])) ht_insert(ht, bits, key_id(pool[s]));
    __syncwarp();
}

// Per-iteration features of the learned stop (definitions in the oracle).
struct FeatState {
    float d1_0, s0, ema;
    int t_last;
};

template <int LW>
__device__ __forceinline__ float pool_dist(const uint64_t (&pool)[LW], int e, int dtype, int metric) {
    uint64_t k = shfl64(pool[0], e & 31);
#pragma unroll
    for (int s = 1; s < LW; s++)
        if ((e >> 5) == s) k = shfl64(pool[s], e & 31);
    uint32_t v = key_to_out((uint32_t)(k >> 32), dtype, metric);
    return dtype == SVF_U8 ? (float)(int32_t)v : __uint_as_float(v);
}

// The top k (k <= 32: slot 0) and, if asked for, the whole final pool.
template <int LW>
__device__ __forceinline__ void write_out(const SearchArgs &a, const uint64_t (&pool)[LW], int lane, int64_t qi) {
    constexpr int L = 32 * LW;
    if (lane < a.k) {
        uint64_t k0 = pool[0];
        bool pad = key_is_pad(k0);
        a.out_ids[qi * a.k + lane] = pad ? kEmpty : key_id(k0);
        a.out_dist[qi * a.k + lane] = key_to_out(pad ? 0xFFFFFFFFu : (uint32_t)(k0 >> 32), a.out_dtype, a.trav.metric);
    }
    if (a.pool_out) {
#pragma unroll
        for (int s = 0; s < LW; s++) {
            uint64_t k0 = pool[s];
            a.pool_out[qi * L + s * 32 + lane] =
                key_is_pad(k0) ? kPad : (k0 & ~(uint64_t)(kExpBit | kNewBit));
        }
    }
}

// The end of a query, warp-wide: the optional exact re-rank of the final
// pool from the primary store, the top k out and the pool out.  False if a
// row copy gave up (SVF_ETIMEOUT recorded).
template <int LW>
__device__ __forceinline__ bool finish_pool(const SearchArgs &a, uint64_t (&pool)[LW], uint32_t *list, uint64_t *keys,
                                            Stage &stg, const float *qf, const uint8_t *qb, int lane, int64_t qi,
                                            int &hits, int &misses) {
    const uint32_t lt_mask = (1u << lane) - 1u;
    // ---- optional exact re-rank of the final pool from the primary store
    if (a.rerank) {
        int npool = 0;
#pragma unroll
        for (int s = 0; s < LW; s++) {
            bool real = !key_is_pad(pool[s]);
            uint32_t b = __ballot_sync(kFull, real);
            if (real) list[npool + __popc(b & lt_mask)] = key_id(pool[s]);
            npool += __popc(b);
        }
        __syncwarp();
        // the fp32 query is still in shared memory
        if (!staged_dist<SVF_F32>(stg, a.prim, list, npool, keys, 0u, lane, qf, qb, a.prim.map ? &a.tier : nullptr,
                                  &hits, &misses)) {
            if (lane == 0) set_error(a.status, SVF_ETIMEOUT, qi);
            return false;
        }
#pragma unroll
        for (int s = 0; s < LW; s++) {
            int e = s * 32 + lane;
            pool[s] = e < npool ? keys[e] : kPad;
        }
        warp_sort<LW>(pool, lane);
    }

    write_out<LW>(a, pool, lane, qi);
    return true;
}

// NCH > 0: the traversal rows are NCH 16-byte chunks (the launcher checks
// the store against it); 0: any layout, read from a.trav at run time.
// VER: graph rows and deletions as of the search's epoch (a.ver), for
// searches that overlap updates in the serving loop; the plain kernel reads
// the current index.
template <int DT, int R, int LW, bool LEARN, int NCH, bool VER>
__global__ void __launch_bounds__(kSearchWarps * 32, SVF_SEARCH_MINB) search_kernel(const SearchArgs a) {
    constexpr int L = 32 * LW;
    constexpr int S = R / 32;  // graph ids per lane
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * kSearchWarps + wib;
    if (qi >= a.nq) return;

    // per warp: query, ids, keys, then the visited table and the staging
    // buffer side by side (the final re-rank stages rows into both)
    uint8_t *my = smem + (size_t)wib * a.warp_smem;
    float *qf = reinterpret_cast<float *>(my);
    uint8_t *qb = my;
    uint32_t *list = reinterpret_cast<uint32_t *>(my + a.q_bytes);
    uint64_t *keys = reinterpret_cast<uint64_t *>(list + a.list_len);
    uint32_t *ht = reinterpret_cast<uint32_t *>(keys + a.list_len);
    Stage stg;
    stg.buf = reinterpret_cast<uint8_t *>(ht + (1 << a.hash_bits));
    stg.cap = a.stage_bytes;
    stg.mbar = reinterpret_cast<uint64_t *>(stg.buf + a.stage_bytes);
    stg.phase[0] = stg.phase[1] = 0;
    if (lane == 0) {
        mbar_init(stg.mbar, 1);
        mbar_init(stg.mbar + 1, 1);
    }

    // ---- query to shared memory, query key
    const uint8_t *qsrc = reinterpret_cast<const uint8_t *>(a.Q) + qi * a.q_row_bytes;
    for (int c = lane; c < a.q_row_bytes / 16; c += 32)
        reinterpret_cast<uint4 *>(my)[c] = __ldg(reinterpret_cast<const uint4 *>(qsrc) + c);
    uint64_t qkey;
    if (a.qkeys) {
        qkey = a.qkeys[qi];
    } else {
        qkey = 0;
        const uint32_t *w = reinterpret_cast<const uint32_t *>(qsrc);
        for (int i = lane; i < a.q_row_bytes / 4; i += 32) qkey += splitmix64(((uint64_t)i << 32) | __ldg(w + i));
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) qkey += shfl64_xor(qkey, m);
    }
    for (int i = lane; i < (1 << a.hash_bits); i += 32) ht[i] = kEmpty;
    __syncwarp();

    // ---- InitCandidatePool: the first L distinct live ids of the draw sequence
    const uint64_t base = splitmix64(a.seed ^ splitmix64(qkey));
    const uint32_t lt_mask = (1u << lane) - 1u;
    int np = 0;
    const int ndraw = 4 * L;
    for (int j0 = 0; j0 < ndraw && np < L && a.n_used > 0; j0 += 32) {
        const int j = j0 + lane;
        // multiply-shift range reduction of the upper 32 random bits
        const uint32_t id = __umulhi((uint32_t)(splitmix64(base ^ (uint64_t)j) >> 32), (uint32_t)a.n_used);
        bool ok = j < ndraw && !(VER ? deleted_at(a.ver, a.del, id) : is_deleted(a.del, id));
        uint32_t m = __match_any_sync(kFull, ok ? id : kEmpty);
        bool first = ok && ((m & lt_mask) == 0);
        bool acc = first && !ht_contains(ht, a.hash_bits, id);
        uint32_t b = __ballot_sync(kFull, acc);
        int rank = __popc(b & lt_mask);
        if (acc && np + rank < L) {
            ht_insert(ht, a.hash_bits, id);
            list[np + rank] = id;
        }
        np += min(__popc(b), L - np);
        __syncwarp();
    }
    int hcount = np;
    const TierCtx *tier = a.trav.map ? &a.tier : nullptr;
    int hits = 0, misses = 0;
    if (!staged_dist<DT, NCH>(stg, a.trav, list, np, keys, 0u, lane, qf, qb, tier, &hits, &misses)) {
        if (lane == 0) set_error(a.status, SVF_ETIMEOUT, qi);
        return;
    }
    uint64_t pool[LW];
#pragma unroll
    for (int s = 0; s < LW; s++) {
        int e = s * 32 + lane;
        pool[s] = e < np ? keys[e] : kPad;
    }
    warp_sort<LW>(pool, lane);

    // learned stop / trace state
    constexpr bool learn = LEARN;
    FeatState fs{0.f, 1.f, 0.f, -1};
    float inv_s0 = 1.f, inv_T = 1.f, inv_k = 1.f;
    if (learn) {
        float d1 = pool_dist<LW>(pool, 0, a.out_dtype, a.trav.metric);
        float dl = pool_dist<LW>(pool, max(np - 1, 0), a.out_dtype, a.trav.metric);
        fs.d1_0 = d1;
        fs.s0 = (dl - d1 > 0.f) ? dl - d1 : 1.f;
        inv_s0 = 1.f / fs.s0;
        inv_T = 1.f / (float)max(a.T, 1);
        inv_k = 1.f / (float)a.k;
    }

    int iters = 0, evals = np, resets = 0, ran = 0;
    const int reset_at = (1 << (a.hash_bits - 1)) - R;
    for (int t = 0; t < a.T; t++) {
        if (hcount > reset_at) {
            ht_reset<LW>(ht, a.hash_bits, pool, lane);
            hcount = 0;
#pragma unroll
            for (int s = 0; s < LW; s++) hcount += __popc(__ballot_sync(kFull, !key_is_pad(pool[s])));
            resets++;
        }
        // GetNearest: the first unexpanded entry in (distance, id) order
        int ps = -1, pl = 0;
#pragma unroll
        for (int s = 0; s < LW; s++) {
            const uint32_t b = __ballot_sync(kFull, ((uint32_t)pool[s] & kExpBit) == 0);
            if (ps < 0 && b) {
                ps = s;
                pl = __ffs(b) - 1;
            }
        }
        if (ps < 0) break;  // nothing left to expand: the pool stays unchanged
        uint32_t pid = 0;
        uint64_t pkey = 0;
#pragma unroll
        for (int s = 0; s < LW; s++)
            if (s == ps) {
                pkey = shfl64(pool[s], pl);
                if (lane == pl) pool[s] |= kExpBit;
            }
        pid = key_id(pkey);
        iters++;

        // FetchNeighbors + filter.  Unvisited ids are staged at once; the
        // deletion bits are read while the rows are in flight and deleted
        // ids are dropped before the merge (putting a deleted id in the
        // visited table changes nothing: it never enters the pool).
        uint32_t nb[S];
        if constexpr (VER) {
            versioned_row<S>(a.ver, a.graph, pid, lane, nb);
        } else {
            const uint32_t *row = a.graph + (int64_t)pid * R;
#pragma unroll
            for (int s = 0; s < S; s++) nb[s] = __ldg(row + s * 32 + lane);
        }
        int nf = 0;
#pragma unroll
        for (int s = 0; s < S; s++) {
            const uint32_t v = nb[s];
            const bool fresh = v != kEmpty && (int64_t)v < a.n_used && ht_insert(ht, a.hash_bits, v);
            const uint32_t b = __ballot_sync(kFull, fresh);
            if (fresh) list[nf + __popc(b & lt_mask)] = v;
            nf += __popc(b);
        }
        hcount += nf;
        __syncwarp();
        uint32_t dword[S];  // deletion-bitset words, consumed after the rows arrive
#pragma unroll
        for (int s = 0; s < S; s++) {
            const int e = s * 32 + lane;
            dword[s] = e < nf ? (VER ? __ldcg(a.del + (list[e] >> 5)) : __ldg(a.del + (list[e] >> 5))) : 0u;
        }
        const uint32_t newflag = learn ? kNewBit : 0u;
        if (!staged_dist<DT, NCH>(stg, a.trav, list, nf, keys, newflag, lane, qf, qb, tier, &hits, &misses)) {
            if (lane == 0) set_error(a.status, SVF_ETIMEOUT, qi);
            return;
        }
        bool dflag[S];
        int ndel = 0;
#pragma unroll
        for (int s = 0; s < S; s++) {
            const int e = s * 32 + lane;
            dflag[s] = e < nf && ((dword[s] >> (list[e] & 31)) & 1u);
            // a deletion after the search's epoch leaves the vertex live for it
            if (VER && dflag[s]) dflag[s] = ld_relaxed_u32(a.ver.del_ep + list[e]) <= a.ver.epoch;
            ndel += __popc(__ballot_sync(kFull, dflag[s]));
        }
        evals += nf - ndel;

        // learned-stop inputs before the merge (only on iterations whose
        // features are used: traced, or where a stop may be taken)
        float d1_prev = 0.f, dk_prev = 0.f;
        const int kk_prev = min(a.k, np);
        const bool evalz = a.mlp != nullptr && t + 1 >= a.t_min && (t + 1 - a.t_min) % a.t_every == 0;
        const bool feats = learn && (a.trace_feat != nullptr || evalz);
        if (feats) {
            d1_prev = pool_dist<LW>(pool, 0, a.out_dtype, a.trav.metric);
            dk_prev = pool_dist<LW>(pool, kk_prev - 1, a.out_dtype, a.trav.metric);
        }

        // only candidates below the pool's current L-th key can enter
        const uint64_t worst = cmpk(shfl64(pool[LW - 1], 31));
        uint64_t cand[S];
        int nin = 0;
#pragma unroll
        for (int s = 0; s < S; s++) {
            const int e = s * 32 + lane;
            cand[s] = (e < nf && !dflag[s]) ? keys[e] : kPad;
            if (cmpk(cand[s]) >= worst) cand[s] = kPad;
            nin += __popc(__ballot_sync(kFull, !key_is_pad(cand[s])));
        }
        nf -= ndel;
        if (nin > 0 && nin <= kFastInsert) {
            // most iterations admit a few candidates: place them directly
            // (the keys buffer is free: the candidates are in registers)
            warp_insert_few<LW, S>(pool, cand, keys, lane);
        } else if (nin > 0) {
            warp_sort<S>(cand, lane);
            if constexpr (S <= LW) {
                warp_merge_into<LW, S>(pool, cand, lane);
            } else {
                // the best L of pool and candidates only need the best L candidates
                uint64_t head[LW];
#pragma unroll
                for (int s = 0; s < LW; s++) head[s] = cand[s];
                warp_merge_into<LW, LW>(pool, head, lane);
            }
        }
        np = min(np + nf, L);
        ran = t + 1;

        if constexpr (LEARN) {
            // newtop: entries of the new top-k admitted in this iteration (an
            // older entry can only move down, so these are exactly the new ids)
            const int kk = min(a.k, np);
            uint32_t bnew = __ballot_sync(kFull, lane < kk && ((uint32_t)pool[0] & kNewBit));
            int newtop = __popc(bnew), admitted = 0, unexp = 0;
#pragma unroll
            for (int s = 0; s < LW; s++) {
                admitted += __popc(__ballot_sync(kFull, ((uint32_t)pool[s] & kNewBit) != 0 && !key_is_pad(pool[s])));
                pool[s] &= ~(uint64_t)kNewBit;
            }
            if (newtop > 0) fs.t_last = t;
            fs.ema = 0.5f * fs.ema + 0.5f * ((float)admitted / R);
            if (!feats) continue;
#pragma unroll
            for (int s = 0; s < LW; s++) unexp += __popc(__ballot_sync(kFull, ((uint32_t)pool[s] & kExpBit) == 0));
            float d1 = pool_dist<LW>(pool, 0, a.out_dtype, a.trav.metric);
            float dk = pool_dist<LW>(pool, kk - 1, a.out_dtype, a.trav.metric);
            float dl = pool_dist<LW>(pool, np - 1, a.out_dtype, a.trav.metric);
            float mine = 0.f;
            if (lane < kk) {
                uint32_t v = key_to_out((uint32_t)(pool[0] >> 32), a.out_dtype, a.trav.metric);
                mine = a.out_dtype == SVF_U8 ? (float)(int32_t)v : __uint_as_float(v);
            }
            float sum = mine;
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) sum += __shfl_xor_sync(kFull, sum, m);
            const float inv_kk = kk == a.k ? inv_k : 1.f / (float)kk;
            const float mean = sum * inv_kk;
            float dev = lane < kk ? (mine - mean) * (mine - mean) : 0.f;
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) dev += __shfl_xor_sync(kFull, dev, m);
            const float inv = inv_s0;
            float f[16];
            f[0] = (float)(t + 1) * inv_T;
            f[1] = (fs.d1_0 - d1) * inv;
            f[2] = (dk - d1) * inv;
            f[3] = (dl - d1) * inv;
            f[4] = (mean - d1) * inv;
            f[5] = sqrtf(dev * inv_kk) * inv;
            f[6] = (float)admitted / R;
            f[7] = (float)unexp / L;
            f[8] = (float)newtop * inv_k;
            f[9] = (float)(t - fs.t_last) * inv_T;
            f[10] = (float)(np - unexp) / L;
            f[11] = (float)(ps * 32 + pl) / L;
            f[12] = (dk_prev - dk) * inv;
            f[13] = (d1_prev - d1) * inv;
            // the next parent: nearest unexpanded entry after the merge
            int ns = -1, nl = 0;
#pragma unroll
            for (int s = 0; s < LW; s++) {
                const uint32_t b = __ballot_sync(kFull, ((uint32_t)pool[s] & kExpBit) == 0);
                if (ns < 0 && b) {
                    ns = s;
                    nl = __ffs(b) - 1;
                }
            }
            const float dnext = ns >= 0 ? pool_dist<LW>(pool, ns * 32 + nl, a.out_dtype, a.trav.metric) : dl;
            f[14] = (dnext - dk) * inv;
            f[15] = fs.ema;
            if (a.trace_feat && lane < 16) {
                float fv = f[0];
#pragma unroll
                for (int i = 1; i < 16; i++)
                    if (lane == i) fv = f[i];
                a.trace_feat[(qi * a.T + t) * 16 + lane] = fv;
            }
            if (evalz) {
                // lane j computes hidden units j and j+32; the packed bf16
                // weights are read through L1 (2.3 KB shared by all warps)
                const uint4 *wp = reinterpret_cast<const uint4 *>(a.mlp);  // W1 rows: 16 bf16 = 2 x uint4
                const uint16_t *wh = reinterpret_cast<const uint16_t *>(a.mlp);
                float z = 0.f;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int j = lane + 32 * h;
                    const uint4 r0 = __ldg(wp + 2 * j), r1 = __ldg(wp + 2 * j + 1);
                    const uint32_t w[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
                    float acc = __uint_as_float((uint32_t)__ldg(wh + kMlpOffB1 + j) << 16);
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        acc = fmaf(__uint_as_float(w[i] << 16), f[2 * i], acc);
                        acc = fmaf(__uint_as_float(w[i] & 0xFFFF0000u), f[2 * i + 1], acc);
                    }
                    if (acc > 0.f) z = fmaf(__uint_as_float((uint32_t)__ldg(wh + kMlpOffW2 + j) << 16), acc, z);
                }
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) z += __shfl_xor_sync(kFull, z, m);
                z += __uint_as_float((uint32_t)__ldg(wh + kMlpOffB2) << 16);
                if (z >= a.z_tau) break;
            }
        }
    }

    // the visited table is no longer needed: the re-rank stages rows into it
    // and the staging buffer after it, so fewer rounds of copies
    stg.buf = reinterpret_cast<uint8_t *>(ht);
    stg.cap = a.stage_bytes + (4u << a.hash_bits);
    if (!finish_pool<LW>(a, pool, list, keys, stg, qf, qb, lane, qi, hits, misses)) return;
    if (a.trace_meta && lane == 0) {
        a.trace_meta[qi * 2 + 0] = ran;
        a.trace_meta[qi * 2 + 1] = fs.t_last;
    }
    if (lane == 0) {
        atomicAdd(a.status + kStQueries, 1ull);
        atomicAdd(a.status + kStIters, (unsigned long long)iters);
        atomicAdd(a.status + kStEvals, (unsigned long long)evals);
        if (resets) atomicAdd(a.status + kStResets, (unsigned long long)resets);
        if (hits | misses) {  // traversal or re-rank rows read through a tiered store
            atomicAdd(a.status + kStHits, (unsigned long long)hits);
            atomicAdd(a.status + kStMisses, (unsigned long long)misses);
        }
    }
}

// Launch search_kernel<DT, R, LW, LEARN, NCH, VER> for a pool of 32 * LW.
template <int DT, int R, bool LEARN, int NCH, bool VER>
cudaError_t launch_search_lw(const SearchArgs &a, int LW, size_t smem, cudaStream_t st) {
    const dim3 grid((unsigned)((a.nq + kSearchWarps - 1) / kSearchWarps)), block(kSearchWarps * 32);
    auto go = [&](auto kernel) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return cudaGetLastError();
        kernel<<<grid, block, smem, st>>>(a);
        return cudaGetLastError();
    };
    switch (LW) {
    case 1: return go(search_kernel<DT, R, 1, LEARN, NCH, VER>);
    case 2: return go(search_kernel<DT, R, 2, LEARN, NCH, VER>);
    case 4: return go(search_kernel<DT, R, 4, LEARN, NCH, VER>);
    case 8: return go(search_kernel<DT, R, 8, LEARN, NCH, VER>);
    }
    return cudaErrorInvalidValue;
}

// The compile-time row layouts of a dtype: d = 96 and d = 128.
template <int DT>
constexpr int nch_for_dim(int d) {
    return d * (DT == SVF_F32 ? 4 : DT == SVF_BF16 ? 2 : 1) / 16;
}
template <int DT, int NCH>
bool layout_is(const RowDesc &r) {
    return r.nchunk == NCH && r.copy_bytes == staged_row_bytes<DT, NCH>() && r.ts == team_for(NCH, DT) &&
           r.cpl == (NCH + team_for(NCH, DT) - 1) / team_for(NCH, DT);
}

// Dispatch on R, learned features, versioned reads and the row layout
// (specialised for the out-degree `RS` at d = 96 and d = 128; everything else
// takes the generic kernel).  Versioned reads run without the learned stop.
template <int DT, int R, int NCH>
cudaError_t launch_search_var(const SearchArgs &a, int LW, bool learn, size_t smem, cudaStream_t st) {
    if (a.ver.row_ver) {
        if (learn) return cudaErrorInvalidValue;
        return launch_search_lw<DT, R, false, NCH, true>(a, LW, smem, st);
    }
    return learn ? launch_search_lw<DT, R, true, NCH, false>(a, LW, smem, st)
                 : launch_search_lw<DT, R, false, NCH, false>(a, LW, smem, st);
}
template <int DT, int RS>
cudaError_t launch_search_dtype(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st) {
    constexpr int N96 = nch_for_dim<DT>(96), N128 = nch_for_dim<DT>(128);
    if (R == RS) {
        if (layout_is<DT, N96>(a.trav)) return launch_search_var<DT, RS, N96>(a, LW, learn, smem, st);
        if (layout_is<DT, N128>(a.trav)) return launch_search_var<DT, RS, N128>(a, LW, learn, smem, st);
    }
    if (R == 32) return launch_search_var<DT, 32, 0>(a, LW, learn, smem, st);
    if (R == 64) return launch_search_var<DT, 64, 0>(a, LW, learn, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace svf
