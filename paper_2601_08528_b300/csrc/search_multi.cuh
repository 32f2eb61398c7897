// search_multi.cuh -- one query per CTA of W warps: the beam search of
// SVFusion Alg. 1 (Sec. 4.2) with the intra-query parallelism of Sec. 4.4
// (several warps serve one query, for small latency-bound batches).
//
// Each iteration expands the W nearest unexpanded pool entries in (distance,
// id) order, one per warp; an id named by several parents is visited once
// (the warps share one visited table in shared memory, and its CAS insert
// decides which warp evaluates the id).  Warp 0 owns the pool (L keys in
// registers) and picks the parents; every warp stages and scores its
// parent's rows and appends the keys that can enter the pool to one shared
// list, which warp 0 merges (one at a time when few, else sorted in groups
// of 32).  Keys are distinct, so the pool is the best L of the old pool and
// all candidates whatever the order of the list.  The initial pool and the
// final re-rank are scored by all warps, a slice each.  W = 1 is the
// one-warp search of search_kernel.cuh.
//
// Shared memory of a CTA: query | visited table | control block | admitted
// keys (W*R) | per warp (candidate ids, keys, row staging buffer, two
// mbarriers).
#pragma once
#include "search_kernel.cuh"

namespace svf {

// Rows ids[0, n) scored by all W warps: warp w takes the w-th slice of
// ceil(n / W) rows into its own keys array.  CTA-wide (ends with a barrier);
// false on every warp if any warp's copies gave up.
template <int DT, int NCH>
__device__ __forceinline__ bool multi_score(Stage &stg, const RowDesc &rd, const uint32_t *ids, int n, uint64_t *keys,
                                            int W, int wid, int lane, const float *qf, const uint8_t *qb,
                                            const TierCtx *tier, int *hits, int *misses, MultiCtl *ctl) {
    const int per = (n + W - 1) / W, i0 = min(wid * per, n), cnt = min(per, n - i0);
    if (!staged_dist<DT, NCH>(stg, rd, ids + i0, cnt, keys, 0u, lane, qf, qb, tier, hits, misses) && lane == 0)
        ctl->abort = 1;
    __syncthreads();
    return !ctl->abort;
}

// Warp 0: the keys of multi_score's slices, sorted, as the pool.
template <int LW, typename KeysOf>
__device__ __forceinline__ void multi_gather(uint64_t (&pool)[LW], int n, int W, KeysOf keys_of, int lane) {
    const int per = (n + W - 1) / W;
#pragma unroll
    for (int s = 0; s < LW; s++) {
        const int e = s * 32 + lane;
        pool[s] = e < n ? keys_of(e / per)[e % per] : kPad;
    }
    warp_sort<LW>(pool, lane);
}

template <int DT, int R, int LW, int NCH, bool VER>
__global__ void __launch_bounds__(kMultiMaxW * 32, 1) search_multi_kernel(const SearchArgs a) {
    constexpr int L = 32 * LW;
    constexpr int S = R / 32;  // graph ids per lane
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int64_t qi = blockIdx.x;
    const uint32_t lt_mask = (1u << lane) - 1u;

    float *qf = reinterpret_cast<float *>(smem);
    uint8_t *qb = smem;
    uint32_t *ht = reinterpret_cast<uint32_t *>(smem + a.q_bytes);
    MultiCtl *ctl = reinterpret_cast<MultiCtl *>(smem + a.q_bytes + ((size_t)4 << a.hash_bits));
    uint64_t *adm = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(ctl) + kMultiCtlBytes);
    uint8_t *warps = reinterpret_cast<uint8_t *>(adm + (size_t)W * R);
    auto list_of = [&](int w) { return reinterpret_cast<uint32_t *>(warps + (size_t)w * a.warp_smem); };
    auto keys_of = [&](int w) { return reinterpret_cast<uint64_t *>(list_of(w) + a.list_len); };
    uint32_t *list = list_of(wid);
    uint64_t *keys = keys_of(wid);
    uint32_t *list0 = list_of(0);  // the lists all warps score: initial pool, re-rank
    Stage stg;
    stg.buf = reinterpret_cast<uint8_t *>(keys + a.list_len);
    stg.cap = a.stage_bytes;
    stg.mbar = reinterpret_cast<uint64_t *>(stg.buf + a.stage_bytes);
    stg.phase[0] = stg.phase[1] = 0;
    if (lane == 0) {
        mbar_init(stg.mbar, 1);
        mbar_init(stg.mbar + 1, 1);
    }

    // ---- query and an empty visited table, by the whole CTA
    const uint8_t *qsrc = reinterpret_cast<const uint8_t *>(a.Q) + qi * a.q_row_bytes;
    for (int c = threadIdx.x; c < a.q_row_bytes / 16; c += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[c] = __ldg(reinterpret_cast<const uint4 *>(qsrc) + c);
    for (int i = threadIdx.x; i < (1 << a.hash_bits); i += blockDim.x) ht[i] = kEmpty;
    if (threadIdx.x == 0) ctl->abort = 0;
    __syncthreads();

    const TierCtx *tier = a.trav.map ? &a.tier : nullptr;
    int hits = 0, misses = 0, iters = 0, evals = 0, resets = 0, hcount = 0, np = 0;
    uint64_t pool[LW];

    // ---- InitCandidatePool: warp 0 draws the first L distinct live ids, all warps score them
    if (wid == 0) {
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
        const uint64_t base = splitmix64(a.seed ^ splitmix64(qkey));
        const int ndraw = 4 * L;
        for (int j0 = 0; j0 < ndraw && np < L && a.n_used > 0; j0 += 32) {
            const int j = j0 + lane;
            const uint32_t id = __umulhi((uint32_t)(splitmix64(base ^ (uint64_t)j) >> 32), (uint32_t)a.n_used);
            bool ok = j < ndraw && !(VER ? deleted_at(a.ver, a.del, id) : is_deleted(a.del, id));
            uint32_t m = __match_any_sync(kFull, ok ? id : kEmpty);
            bool first = ok && ((m & lt_mask) == 0);
            bool acc = first && !ht_contains(ht, a.hash_bits, id);
            uint32_t b = __ballot_sync(kFull, acc);
            int rank = __popc(b & lt_mask);
            if (acc && np + rank < L) {
                ht_insert(ht, a.hash_bits, id);
                list0[np + rank] = id;
            }
            np += min(__popc(b), L - np);
            __syncwarp();
        }
        hcount = evals = np;
        if (lane == 0) ctl->nrows = np;
    }
    __syncthreads();
    if (!multi_score<DT, NCH>(stg, a.trav, list0, ctl->nrows, keys, W, wid, lane, qf, qb, tier, &hits, &misses, ctl)) {
        if (wid == 0 && lane == 0) set_error(a.status, SVF_ETIMEOUT, qi);
        return;
    }
    if (wid == 0) multi_gather<LW>(pool, np, W, keys_of, lane);

    const int reset_at = (1 << (a.hash_bits - 1)) - W * R;
    for (int t = 0; t < a.T; t++) {
        // ---- warp 0: the W nearest unexpanded entries become this iteration's parents
        if (wid == 0) {
            if (hcount > reset_at) {
                ht_reset<LW>(ht, a.hash_bits, pool, lane);
                hcount = 0;
#pragma unroll
                for (int s = 0; s < LW; s++) hcount += __popc(__ballot_sync(kFull, !key_is_pad(pool[s])));
                resets++;
            }
            int before = 0;
#pragma unroll
            for (int s = 0; s < LW; s++) {
                const bool un = ((uint32_t)pool[s] & kExpBit) == 0;  // pads carry the bit
                const uint32_t b = __ballot_sync(kFull, un);
                const int rank = before + __popc(b & lt_mask);
                if (un && rank < W) {
                    ctl->par[rank] = key_id(pool[s]);
                    pool[s] |= kExpBit;
                }
                before += __popc(b);
            }
            const uint64_t worst = cmpk(shfl64(pool[LW - 1], 31));
            if (lane == 0) {
                ctl->npar = min(before, W);
                ctl->worst = worst;
                ctl->nadm = ctl->nf = ctl->nlive = 0;
            }
            iters += min(before, W);
        }
        __syncthreads();
        const int npar = ctl->npar;
        if (npar == 0) break;  // nothing left to expand: the pool stays unchanged

        // ---- warp w < npar: FetchNeighbors of parent w, filter, stage, score,
        //      append the keys that can enter the pool
        if (wid < npar) {
            uint32_t nb[S];
            if constexpr (VER) {
                versioned_row<S>(a.ver, a.graph, ctl->par[wid], lane, nb);
            } else {
                const uint32_t *row = a.graph + (int64_t)ctl->par[wid] * R;
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
            __syncwarp();
            uint32_t dword[S];
#pragma unroll
            for (int s = 0; s < S; s++) {
                const int e = s * 32 + lane;
                dword[s] = e < nf ? (VER ? __ldcg(a.del + (list[e] >> 5)) : __ldg(a.del + (list[e] >> 5))) : 0u;
            }
            if (!staged_dist<DT, NCH>(stg, a.trav, list, nf, keys, 0u, lane, qf, qb, tier, &hits, &misses)) {
                if (lane == 0) {
                    set_error(a.status, SVF_ETIMEOUT, qi);
                    ctl->abort = 1;
                }
                nf = 0;
            }
            // deleted ids and keys at or above the pool's L-th key cannot enter
            const uint64_t worst = ctl->worst;
            int nlive = 0, nin = 0;
            uint64_t cand[S];
#pragma unroll
            for (int s = 0; s < S; s++) {
                const int e = s * 32 + lane;
                bool live = e < nf && !((dword[s] >> (list[e] & 31)) & 1u);
                // a deletion after the search's epoch leaves the vertex live for it
                if (VER && e < nf && !live) live = ld_relaxed_u32(a.ver.del_ep + list[e]) > a.ver.epoch;
                nlive += __popc(__ballot_sync(kFull, live));
                cand[s] = live ? keys[e] : kPad;
                if (cmpk(cand[s]) >= worst) cand[s] = kPad;
                nin += __popc(__ballot_sync(kFull, !key_is_pad(cand[s])));
            }
            int at = 0;
            if (lane == 0) {
                at = nin ? atomicAdd(&ctl->nadm, nin) : 0;
                atomicAdd(&ctl->nf, nf);
                atomicAdd(&ctl->nlive, nlive);
            }
            at = __shfl_sync(kFull, at, 0);
#pragma unroll
            for (int s = 0; s < S; s++) {
                const bool in = !key_is_pad(cand[s]);
                const uint32_t b = __ballot_sync(kFull, in);
                if (in) adm[at + __popc(b & lt_mask)] = cand[s];
                at += __popc(b);
            }
        }
        __syncthreads();
        if (ctl->abort) return;

        // ---- warp 0: merge the admitted keys into the pool
        if (wid == 0) {
            const int nadm = ctl->nadm;
            hcount += ctl->nf;
            evals += ctl->nlive;
            np = min(np + ctl->nlive, L);
            if (nadm <= kFastInsert) {
                for (int i = 0; i < nadm; i++) warp_insert_one<LW>(pool, adm[i], lane);
            } else {
                for (int i0 = 0; i0 < nadm; i0 += 32) {
                    uint64_t cand[1] = {i0 + lane < nadm ? adm[i0 + lane] : kPad};
                    warp_sort<1>(cand, lane);
                    warp_merge_into<LW, 1>(pool, cand, lane);
                }
            }
        }
    }

    // ---- optional exact re-rank, every warp a slice of the final pool; outputs
    if (a.rerank) {
        if (wid == 0) {
            int npool = 0;
#pragma unroll
            for (int s = 0; s < LW; s++) {
                const bool real = !key_is_pad(pool[s]);
                const uint32_t b = __ballot_sync(kFull, real);
                if (real) list0[npool + __popc(b & lt_mask)] = key_id(pool[s]);
                npool += __popc(b);
            }
            if (lane == 0) ctl->nrows = npool;
        }
        __syncthreads();
        const int npool = ctl->nrows;
        if (!multi_score<SVF_F32, 0>(stg, a.prim, list0, npool, keys, W, wid, lane, qf, qb,
                                     a.prim.map ? &a.tier : nullptr, &hits, &misses, ctl)) {
            if (wid == 0 && lane == 0) set_error(a.status, SVF_ETIMEOUT, qi);
            return;
        }
        if (wid == 0) multi_gather<LW>(pool, npool, W, keys_of, lane);
    }
    if (wid == 0) write_out<LW>(a, pool, lane, qi);
    if (lane == 0) {
        if (wid == 0) {
            atomicAdd(a.status + kStQueries, 1ull);
            atomicAdd(a.status + kStIters, (unsigned long long)iters);
            atomicAdd(a.status + kStEvals, (unsigned long long)evals);
            if (resets) atomicAdd(a.status + kStResets, (unsigned long long)resets);
        }
        if (hits | misses) {  // traversal or re-rank rows read through a tiered store
            atomicAdd(a.status + kStHits, (unsigned long long)hits);
            atomicAdd(a.status + kStMisses, (unsigned long long)misses);
        }
    }
}

// Launch search_multi_kernel for W warps per query and a pool of 32 * LW.
template <int DT, int R, int NCH, bool VER>
cudaError_t launch_multi_lw(const SearchArgs &a, int W, int LW, size_t smem, cudaStream_t st) {
    const dim3 grid((unsigned)a.nq), block((unsigned)(32 * W));
    auto go = [&](auto kernel) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return cudaGetLastError();
        kernel<<<grid, block, smem, st>>>(a);
        return cudaGetLastError();
    };
    switch (LW) {
    case 1: return go(search_multi_kernel<DT, R, 1, NCH, VER>);
    case 2: return go(search_multi_kernel<DT, R, 2, NCH, VER>);
    case 4: return go(search_multi_kernel<DT, R, 4, NCH, VER>);
    case 8: return go(search_multi_kernel<DT, R, 8, NCH, VER>);
    }
    return cudaErrorInvalidValue;
}

// Dispatch on R, versioned reads and the row layout, as launch_search_dtype does.
template <int DT, int R, int NCH>
cudaError_t launch_multi_var(const SearchArgs &a, int W, int LW, size_t smem, cudaStream_t st) {
    return a.ver.row_ver ? launch_multi_lw<DT, R, NCH, true>(a, W, LW, smem, st)
                         : launch_multi_lw<DT, R, NCH, false>(a, W, LW, smem, st);
}
template <int DT, int RS>
cudaError_t launch_multi_dtype(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st) {
    constexpr int N96 = nch_for_dim<DT>(96), N128 = nch_for_dim<DT>(128);
    if (R == RS) {
        if (layout_is<DT, N96>(a.trav)) return launch_multi_var<DT, RS, N96>(a, W, LW, smem, st);
        if (layout_is<DT, N128>(a.trav)) return launch_multi_var<DT, RS, N128>(a, W, LW, smem, st);
    }
    if (R == 32) return launch_multi_var<DT, 32, 0>(a, W, LW, smem, st);
    if (R == 64) return launch_multi_var<DT, 64, 0>(a, W, LW, smem, st);
    return cudaErrorInvalidValue;
}

}  // namespace svf
