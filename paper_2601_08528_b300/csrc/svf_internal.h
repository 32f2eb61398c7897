// svf_internal.h -- launch interfaces shared by the .cu files of libsvf.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/svf.h"
#include "svf_dev.cuh"

namespace svf {

// SMs of the current device (148 on a B300 when no device can be queried,
// e.g. sizing scratch on a host without a GPU).
inline int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0) {
        cudaGetLastError();
        return 148;
    }
    return n;
}

constexpr int kSearchWarps = 4;  // queries (warps) per CTA

// Several warps per query (search_multi.cuh): W parents per iteration.
constexpr int kMultiMaxW = 8;
struct MultiCtl {
    uint32_t par[kMultiMaxW];  // this iteration's parents, nearest first
    uint64_t worst;            // the pool's L-th key (flags masked) before the merge
    int npar;
    int nadm;                  // admitted keys appended this iteration
    int nf;                    // ids staged this iteration (fresh, deletions included)
    int nlive;                 // of them, not deleted
    int nrows;                 // rows of a list scored by all warps (initial pool, re-rank)
    int abort;                 // a row copy gave up: every warp leaves
};
constexpr size_t kMultiCtlBytes = (sizeof(MultiCtl) + 15) / 16 * 16;

struct SearchArgs {
    RowDesc trav;  // store read by the traversal
    RowDesc prim;  // primary store (exact re-rank)
    const uint32_t *graph;
    const uint32_t *del;
    int64_t n_used;
    const void *Q;
    int64_t nq;
    int q_row_bytes;  // bytes of one query row (d*4, or d for U8)
    int q_bytes;      // shared-memory bytes reserved for the query
    const uint64_t *qkeys;
    uint64_t seed;
    int k, T;
    int hash_bits;
    int rerank;
    int out_dtype;    // SVF_U8 -> int32 distances, else float
    uint32_t *out_ids;
    uint32_t *out_dist;
    uint64_t *pool_out;
    const void *mlp;
    float z_tau;
    int t_min;
    int t_every;
    float *trace_feat;
    int32_t *trace_meta;
    unsigned long long *status;
    TierCtx tier;     // tiered store (used when trav.map is set)
    int list_len;
    uint32_t stage_bytes;
    size_t warp_smem;
    int W;            // warps (parents per iteration) per query; 1: one warp per query
    VerCtx ver;       // versioned reads (searches overlapping updates), or ver.row_ver == null
};

cudaError_t launch_search(SearchArgs a, int R, int L, cudaStream_t st);

// Brute-force exact kNN over the rows of a store (knn.cu).
struct KnnArgs {
    RowDesc X;        // database rows [0, n)
    int64_t n;
    const void *Q;    // query rows: fp32 [nq][d] or uint8 for U8
    int q_row_bytes;
    int64_t nq;
    const int64_t *self;   // skip this id per query (device) or null
    int64_t self_base;     // if self is null and >= 0: query i skips id self_base + i
    const uint32_t *del;   // skip deleted (device) or null
    int k;                 // <= 128
    uint64_t *out_keys;    // [nq][k] sorted keys (PAD-filled)
    // Optional scratch for small batches: with it, the rows are split into
    // slices scanned by separate blocks (one block per 32 queries would leave
    // most SMs idle), each slice's exact top k lands here and a merge keeps
    // the best k of each query.  Null: one block per 32 queries scans every row.
    uint64_t *part_keys;
    size_t part_bytes;
};
cudaError_t launch_knn(const KnnArgs &a, cudaStream_t st);
// Same, with queries taken from the store itself (rows q0 .. q0+nq-1),
// excluding each query's own row.
cudaError_t launch_knn_self(const RowDesc &X, int64_t n, int64_t q0, int64_t nq, int k, uint64_t *out_keys,
                            cudaStream_t st);

// Keys -> (ids, dists) output arrays.
cudaError_t launch_keys_to_out(const uint64_t *keys, int64_t nq, int kin, int kout, int dtype, int metric,
                               uint32_t *ids, uint32_t *dist, cudaStream_t st);

// Neighbour reordering (prune.cu).  For each vertex v_i (i < nv) the sorted
// candidate keys cand[i][0..ncand) (PAD-terminated) are reordered into
// out_rows[i][0..R).  nbr: graph rows consulted by RANK (width nbr_w).
constexpr int kPruneStageBytes = 160 * 1024;  // candidate rows the prune stages in shared memory

struct PruneArgs {
    RowDesc X;
    const uint64_t *cand;
    int cand_stride;
    int64_t nv;
    const uint32_t *vids;   // vertex id of each list (null: vids[i] = v0 + i)
    int64_t v0;
    int mode;
    const uint32_t *nbr;
    int nbr_w;
    int R;
    uint32_t *out_rows;     // [nv][R]
    uint32_t *out_dkey;     // [nv][R] distance key of each chosen entry (may be null)
    const int32_t *count;   // device count of lists (null: nv)
};
cudaError_t launch_prune(const PruneArgs &a, int max_lists, cudaStream_t st);

// Encoders (codec.cu).
cudaError_t launch_encode_bf16(const float *X, int64_t n, int d, uint16_t *out, cudaStream_t st);
cudaError_t launch_encode_fp8(const float *X, int64_t n, int d, uint8_t *out, int64_t pitch, cudaStream_t st);

}  // namespace svf
