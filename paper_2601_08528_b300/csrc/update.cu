// update.cu -- index updates of SVFusion on the GPU (Sec. 5):
//   insert: reverse-edge patch of the tail half of every chosen neighbour
//           (requests grouped per target through an atomic linked list, then
//           merged deterministically by (distance, id));
//   delete: bitset marking with validation, detection of vertices whose
//           out-neighbours are more than half deleted, and the candidate
//           gathering of the localized repair (at most c entries from each
//           deleted neighbour's list), all from a snapshot of the rows;
//   codecs: fp32 -> bfloat16 / FP8-E4M3 with a per-vector scale.
#include <cstdint>

#include "svf_internal.h"
#include "svf_update.h"

namespace svf {

// ---------------------------------------------------------------- insert
__global__ void rev_link_kernel(const uint32_t *rows, int64_t nreq, int64_t tmax, int32_t *head, int32_t *next) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nreq) return;
    uint32_t u = rows[i];
    if (u == kEmpty || (int64_t)u >= tmax) return;
    next[i] = atomicExch(head + u, (int32_t)i);
}

// One warp per request; the request that ended up at the head of its
// target's list owns the target and rewrites the target's tail half.
template <int DT>
__global__ void rev_merge_kernel(const RowDesc X, uint32_t *graph, int R, const uint32_t *del, int64_t n0,
                                 const uint32_t *rows, const uint32_t *dkeys, int64_t nreq, int64_t tmax,
                                 const int32_t *head, const int32_t *next, unsigned long long *status) {
    const int lane = threadIdx.x & 31, sub = lane & 7, team = lane >> 3;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= nreq) return;
    const uint32_t u = rows[i];
    if (u == kEmpty || (int64_t)u >= tmax || head[u] != (int32_t)i) return;
    const int H = R / 2, TL = R - R / 2;
    uint32_t *row = graph + (int64_t)u * R;
    // live tail entries with their distances to u
    uint32_t t = lane < TL ? row[H + lane] : kEmpty;
    bool live = t != kEmpty && (int64_t)t < n0 && !is_deleted(del, t);
    uint64_t best[1] = {kPad};
    const uint4 *ru = reinterpret_cast<const uint4 *>(row_ptr(X, u));
    for (int b = 0; b < TL; b += 4) {
        const int e = b + team;  // entry evaluated by this team
        const uint32_t te = __shfl_sync(kFull, t, e & 31);
        const bool le = __shfl_sync(kFull, live, e & 31) && e < TL;
        const uint4 *rt = reinterpret_cast<const uint4 *>(row_ptr(X, le ? te : u));
        const uint32_t key = team_pair_key<DT>(X.metric, ru, rt, le ? X.nchunk : 0, sub);
        const uint64_t full = le ? make_key(key, te) : kPad;
        // entry b+s is held by the lanes of team s; bring it to lane b+s
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const uint64_t v = shfl64(full, s * 8);
            if (lane == b + s) best[0] = v;
        }
    }
    warp_sort<1>(best, lane);
    // requests, 32 at a time, in list order (the merged result does not
    // depend on that order); `cur` is the same on every lane
    int32_t cur = head[u];
    while (cur >= 0) {
        int32_t mine = -1;
        for (int j = 0; j < 32 && cur >= 0; j++) {
            if (lane == j) mine = cur;
            cur = next[cur];
        }
        uint64_t ck[1] = {kPad};
        if (mine >= 0) ck[0] = make_key(dkeys[mine], (uint32_t)(n0 + mine / R));
        warp_sort<1>(ck, lane);
        warp_merge_into<1, 1>(best, ck, lane);
    }
    if (lane < TL) row[H + lane] = key_is_pad(best[0]) ? kEmpty : key_id(best[0]);
    if (lane == 0) atomicAdd(status + kStRevTargets, 1ull);
}

// Copy row u into the next shadow row of the update, point u at it, then
// stamp u with the update's number (release: the copy and the pointer are
// visible before the stamp, and the stamp before any later kernel of the
// update rewrites the row).
__device__ __forceinline__ void stamp_row(const uint32_t *graph, int R, uint32_t u, const VerUpd &v,
                                          unsigned long long *status) {
    const unsigned long long k = atomicAdd(v.counter, 1ull);
    if ((int64_t)k >= v.cap) {  // the caller sized the half for the update: a guard only
        set_error(status, SVF_ECAPACITY, (long long)u);
        return;
    }
    const int64_t slot = v.base + (int64_t)k;
    for (int r = 0; r < R; r++) v.shadow[slot * R + r] = graph[(int64_t)u * R + r];
    v.shadow_slot[u] = (int32_t)slot;
    __threadfence();
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(v.row_ver + u), "r"(v.E) : "memory");
}

// One thread per request; the request at the head of its target's list
// stamps the target (each target once).
__global__ void stamp_targets_kernel(const uint32_t *graph, int R, const uint32_t *rows, int64_t nreq, int64_t tmax,
                                     const int32_t *head, VerUpd v, unsigned long long *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nreq) return;
    const uint32_t u = rows[i];
    if (u == kEmpty || (int64_t)u >= tmax || head[u] != (int32_t)i) return;
    stamp_row(graph, R, u, v, status);
}

__global__ void stamp_rows_kernel(const uint32_t *graph, int R, const uint32_t *vl, int64_t nv, VerUpd v,
                                  unsigned long long *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) stamp_row(graph, R, vl[i], v, status);
}

cudaError_t launch_stamp_rows(const uint32_t *graph, int R, const uint32_t *vl, int64_t nv, const VerUpd &ver,
                              unsigned long long *status, cudaStream_t st) {
    if (nv == 0) return cudaSuccess;
    stamp_rows_kernel<<<(unsigned)((nv + 127) / 128), 128, 0, st>>>(graph, R, vl, nv, ver, status);
    return cudaGetLastError();
}

__global__ void rev_reset_kernel(const uint32_t *rows, int64_t nreq, int64_t tmax, int32_t *head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nreq) return;
    uint32_t u = rows[i];
    if (u != kEmpty && (int64_t)u < tmax) head[u] = -1;
}

__global__ void iota_kernel(uint32_t *out, int64_t m, int64_t base) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = (uint32_t)(base + i);
}

cudaError_t launch_reverse_patch(const RowDesc &X, uint32_t *graph, int R, const uint32_t *del, int64_t n0, int64_t m,
                                 const uint32_t *rows, const uint32_t *dkeys, int64_t tmax, int32_t *head,
                                 int32_t *next, unsigned long long *status, cudaStream_t st, const VerUpd *ver) {
    const int64_t nreq = m * R;
    if (nreq == 0) return cudaSuccess;
    rev_link_kernel<<<(unsigned)((nreq + 255) / 256), 256, 0, st>>>(rows, nreq, tmax, head, next);
    if (ver)
        stamp_targets_kernel<<<(unsigned)((nreq + 255) / 256), 256, 0, st>>>(graph, R, rows, nreq, tmax, head, *ver,
                                                                             status);
    const unsigned g = (unsigned)((nreq * 32 + 255) / 256);
    if (X.dtype == SVF_U8)
        rev_merge_kernel<SVF_U8><<<g, 256, 0, st>>>(X, graph, R, del, n0, rows, dkeys, nreq, tmax, head, next, status);
    else
        rev_merge_kernel<SVF_F32><<<g, 256, 0, st>>>(X, graph, R, del, n0, rows, dkeys, nreq, tmax, head, next,
                                                     status);
    rev_reset_kernel<<<(unsigned)((nreq + 255) / 256), 256, 0, st>>>(rows, nreq, tmax, head);
    return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t *out, int64_t m, int64_t base, cudaStream_t st) {
    if (m == 0) return cudaSuccess;
    iota_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(out, m, base);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- delete
__global__ void del_validate_kernel(const uint32_t *ids, int64_t m, int64_t n_used, unsigned long long *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    if ((int64_t)ids[i] >= n_used) atomicCAS(status + kStScratch0, 0ull, (unsigned long long)i + 1ull);
}

__global__ void del_mark_kernel(const uint32_t *ids, int64_t m, uint32_t *del, unsigned long long *status,
                                long long *out_newly, uint32_t *del_ep, uint32_t E) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || status[kStScratch0] != 0ull) return;
    const uint32_t id = ids[i], bit = 1u << (id & 31);
    if (del_ep) {
        // the deletion's number first (a vertex already deleted keeps its own)
        atomicMin(del_ep + id, E);
        __threadfence();
    }
    const uint32_t old = atomicOr(del + (id >> 5), bit);
    if (!(old & bit)) {
        atomicAdd(status + kStNewlyDeleted, 1ull);
        atomicAdd(status + kStScratch0 + 1, 1ull);
    }
}

// Warp per row: live rows with at least min_del deleted entries join V^L
// (the localized repair: more than R/2; global consolidation: 1).
__global__ void del_scan_kernel(const uint32_t *graph, int R, const uint32_t *del, int64_t n_used, int min_del,
                                uint32_t *vl, unsigned long long *status) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (status[kStScratch0] != 0ull) return;
    for (int64_t u = w0; u < n_used; u += nw) {
        if (is_deleted(del, (uint32_t)u)) continue;
        int nd = 0;
        for (int s = 0; s < R; s += 32) {
            uint32_t t = graph[u * R + s + lane];
            nd += __popc(__ballot_sync(kFull, t != kEmpty && is_deleted(del, t)));
        }
        if (nd >= min_del && lane == 0) {
            unsigned long long p = atomicAdd(status + kStScratch0 + 2, 1ull);
            vl[p] = (uint32_t)u;
        }
    }
}

// Warp per V^L vertex: candidate list (live row entries, then the first c
// new live entries of each deleted neighbour's row, at most cap in all;
// cap >= R), distances, sorted keys.
template <int DT>
__global__ void del_gather_kernel(const RowDesc X, const uint32_t *graph, int R, const uint32_t *del, int64_t n_used,
                                  int c, int cap, const uint32_t *vl, int64_t v0, int64_t nv, uint64_t *cand,
                                  int cstride) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, team = lane >> 3, sub = lane & 7;
    const int HB = 10;  // 1024-slot id table per warp (<= 512 candidates)
    uint32_t *ht = reinterpret_cast<uint32_t *>(sm) + wib * ((1 << HB) + 2 * kMaxRepair);
    uint32_t *list = ht + (1 << HB);
    uint32_t *dks = list + kMaxRepair;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= nv) return;
    const uint32_t u = vl[v0 + i];
    const uint32_t lt = (1u << lane) - 1u;
    for (int e = lane; e < (1 << HB); e += 32) ht[e] = kEmpty;
    __syncwarp();
    auto ht_has = [&](uint32_t id) {
        uint32_t h = (id * 0x9E3779B1u) >> (32 - HB);
        for (int p = 0; p < (1 << HB); p++) {
            uint32_t v = ht[h];
            if (v == id) return true;
            if (v == kEmpty) return false;
            h = (h + 1) & ((1u << HB) - 1u);
        }
        return false;
    };
    auto ht_put = [&](uint32_t id) {
        uint32_t h = (id * 0x9E3779B1u) >> (32 - HB);
        for (int p = 0; p < (1 << HB); p++) {
            uint32_t old = atomicCAS(ht + h, kEmpty, id);
            if (old == kEmpty || old == id) return;
            h = (h + 1) & ((1u << HB) - 1u);
        }
    };
    const uint32_t *row = graph + (int64_t)u * R;
    int n = 0;
    for (int s = 0; s < R; s += 32) {
        uint32_t t = row[s + lane];
        bool ok = t != kEmpty && (int64_t)t < n_used && !is_deleted(del, t) && t != u;
        uint32_t mm = __match_any_sync(kFull, ok ? t : kEmpty);
        ok = ok && (mm & lt) == 0 && !ht_has(t);
        uint32_t b = __ballot_sync(kFull, ok);
        if (ok) {
            ht_put(t);
            list[n + __popc(b & lt)] = t;
        }
        n += __popc(b);
        __syncwarp();
    }
    for (int e = 0; e < R; e++) {
        const uint32_t p = row[e];
        if (p == kEmpty || (int64_t)p >= n_used || !is_deleted(del, p)) continue;
        const uint32_t *prow = graph + (int64_t)p * R;
        int taken = 0;
        for (int s = 0; s < R && taken < c && n < cap; s += 32) {
            uint32_t w = prow[s + lane];
            bool ok = w != kEmpty && (int64_t)w < n_used && !is_deleted(del, w) && w != u;
            uint32_t mm = __match_any_sync(kFull, ok ? w : kEmpty);
            ok = ok && (mm & lt) == 0 && !ht_has(w);
            uint32_t b = __ballot_sync(kFull, ok);
            int rk = __popc(b & lt);
            if (ok && taken + rk < c && n + rk < cap) {
                ht_put(w);
                list[n + rk] = w;
            }
            int add = min(__popc(b), min(c - taken, cap - n));
            n += add;
            taken += add;
            __syncwarp();
        }
    }
    __syncwarp();
    // distances to u (teams of 8)
    const uint4 *ru = reinterpret_cast<const uint4 *>(row_ptr(X, u));
    for (int b0 = 0; b0 < n; b0 += 4) {
        const int e = b0 + team;
        const bool ve = e < n;
        const uint32_t w = ve ? list[e] : u;
        const uint4 *rw = reinterpret_cast<const uint4 *>(row_ptr(X, w));
        uint32_t key = team_pair_key<DT>(X.metric, ru, rw, ve ? X.nchunk : 0, sub);
        if (ve && sub == 0) dks[e] = key;
    }
    __syncwarp();
    // rank sort by (distance, id)
    uint64_t *out = cand + i * cstride;
    for (int e = lane; e < n; e += 32) {
        const uint64_t ke = make_key(dks[e], list[e]);
        int pos = 0;
        for (int f = 0; f < n; f++) pos += make_key(dks[f], list[f]) < ke;
        out[pos] = ke;
    }
    for (int e = n + lane; e < cstride; e += 32) out[e] = kPad;
}

// One thread per V^L vertex: new row = pruned row, then u's deleted
// entries in their old order fill the slots the prune left empty.
__global__ void del_finalize_kernel(uint32_t *graph, int R, const uint32_t *del, const uint32_t *vl, int64_t nv,
                                    const uint32_t *newrows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    uint32_t *row = graph + (int64_t)vl[i] * R;
    const uint32_t *nr = newrows + i * R;
    uint32_t buf[64];
    int w = 0;
    for (int r = 0; r < R; r++) {
        buf[r] = nr[r];
        w += nr[r] != kEmpty;
    }
    for (int r = 0; r < R && w < R; r++) {
        const uint32_t t = row[r];
        if (t != kEmpty && is_deleted(del, t)) buf[w++] = t;
    }
    for (int r = 0; r < R; r++) row[r] = buf[r];
}

cudaError_t launch_delete_mark(const uint32_t *ids, int64_t m, int64_t n_used, uint32_t *del,
                               unsigned long long *status, cudaStream_t st, const VerUpd *ver) {
    if (m == 0) return cudaSuccess;
    const unsigned g = (unsigned)((m + 255) / 256);
    del_validate_kernel<<<g, 256, 0, st>>>(ids, m, n_used, status);
    del_mark_kernel<<<g, 256, 0, st>>>(ids, m, del, status, nullptr, ver ? ver->del_ep : nullptr, ver ? ver->E : 0u);
    return cudaGetLastError();
}

cudaError_t launch_delete_scan(const uint32_t *graph, int R, const uint32_t *del, int64_t n_used, int min_del,
                               uint32_t *vl, unsigned long long *status, cudaStream_t st) {
    if (n_used == 0) return cudaSuccess;
    const int64_t cap = (int64_t)sm_count() * 64;
    int64_t warps = n_used < cap ? n_used : cap;
    del_scan_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(graph, R, del, n_used, min_del, vl,
                                                                            status);
    return cudaGetLastError();
}

cudaError_t launch_delete_gather(const RowDesc &X, const uint32_t *graph, int R, const uint32_t *del, int64_t n_used,
                                 int c, int cap, const uint32_t *vl, int64_t v0, int64_t nv, uint64_t *cand,
                                 int cstride, cudaStream_t st) {
    if (nv == 0) return cudaSuccess;
    const int wpb = 4;
    const size_t smem = (size_t)wpb * ((1 << 10) + 2 * kMaxRepair) * 4;
    const unsigned g = (unsigned)((nv + wpb - 1) / wpb);
    if (X.dtype == SVF_U8) {
        cudaFuncSetAttribute(del_gather_kernel<SVF_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        del_gather_kernel<SVF_U8><<<g, wpb * 32, smem, st>>>(X, graph, R, del, n_used, c, cap, vl, v0, nv, cand,
                                                              cstride);
    } else {
        cudaFuncSetAttribute(del_gather_kernel<SVF_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        del_gather_kernel<SVF_F32><<<g, wpb * 32, smem, st>>>(X, graph, R, del, n_used, c, cap, vl, v0, nv, cand,
                                                               cstride);
    }
    return cudaGetLastError();
}

cudaError_t launch_delete_finalize(uint32_t *graph, int R, const uint32_t *del, const uint32_t *vl, int64_t nv,
                                   const uint32_t *newrows, cudaStream_t st) {
    if (nv == 0) return cudaSuccess;
    del_finalize_kernel<<<(unsigned)((nv + 127) / 128), 128, 0, st>>>(graph, R, del, vl, nv, newrows);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- codecs
__global__ void enc_bf16_kernel(const float *X, int64_t n, uint16_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    __nv_bfloat16 h = __float2bfloat16_rn(X[i]);
    out[i] = *reinterpret_cast<uint16_t *>(&h);
}

// Warp per row: s = max|x| / 448 (1 if 0), code_i = E4M3(x_i / s), satfinite.
__global__ void enc_fp8_kernel(const float *X, int64_t n, int d, uint8_t *out, int64_t pitch) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    const float *x = X + r * d;
    float mx = 0.f;
    for (int i = lane; i < d; i += 32) mx = fmaxf(mx, fabsf(x[i]));
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, m));
    const float s = mx == 0.f ? 1.f : __fdiv_rn(mx, 448.f);
    uint8_t *o = out + r * pitch;
    for (int i = lane; i < d; i += 32) o[i] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(x[i], s), __NV_SATFINITE, __NV_E4M3);
    if (lane == 0) *reinterpret_cast<float *>(o + d) = s;
    for (int i = d + 4 + lane; i < pitch; i += 32) o[i] = 0;
}

cudaError_t launch_encode_bf16(const float *X, int64_t n, int d, uint16_t *out, cudaStream_t st) {
    int64_t e = n * d;
    if (e == 0) return cudaSuccess;
    enc_bf16_kernel<<<(unsigned)((e + 255) / 256), 256, 0, st>>>(X, e, out);
    return cudaGetLastError();
}

cudaError_t launch_encode_fp8(const float *X, int64_t n, int d, uint8_t *out, int64_t pitch, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    enc_fp8_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(X, n, d, out, pitch);
    return cudaGetLastError();
}

}  // namespace svf
