// index_impl.h -- the host-side index object behind the C ABI (shared by
// api.cu and tier.cu): parameters, borrowed buffers, workspace layout, and
// the row descriptors of the stores.
#pragma once
#include <cmath>
#include <functional>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "svf_internal.h"
#include "svf_update.h"

namespace svf {

int fail(int code, const char *fmt, ...);

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess) return svf::fail(SVF_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline int esize_of(int dtype) { return dtype == SVF_U8 ? 1 : 4; }
inline int64_t fp8_pitch(int d) { return ((int64_t)d + 4 + 31) / 32 * 32; }

// Lanes per row when distances are computed from staged rows: the smallest
// power of two that leaves at most max_chunks_per_lane(dtype) chunks of 16
// bytes per lane (8 for FP8 rows, 4 otherwise).
inline void set_team(RowDesc &r) {
    int ts = 1;
    while (ts < 32 && (r.nchunk + ts - 1) / ts > max_chunks_per_lane(r.dtype)) ts <<= 1;
    r.ts = ts;
    r.cpl = (r.nchunk + ts - 1) / ts;
}

// Exact 2R-NN of the build on the tensor cores (tc_knn.cu): used for fp32
// inner-product stores and uint8 stores with d <= 128, 2R <= 128 and at least
// 2^16 rows; scratch inside the workspace.
bool tc_build_applies(int dtype, int metric, int d, int64_t n, int K);
size_t tc_build_scratch_bytes(int64_t n, int d, int K);
int tc_build_knn(const RowDesc &X, int64_t n, int K, uint8_t *scratch, size_t bytes, uint64_t *keys,
                 int64_t *out_fallback, cudaStream_t st);

struct WsLayout {
    size_t head, vl, newrows, region, total;
    size_t knn_keys, knn_ids;        // build
    size_t tc, tc_bytes;             // build on the tensor cores
    size_t pool, rows, dkeys, next;  // insert
    size_t cand;                     // delete
    int64_t max_batch;
};

constexpr int kInsertLmax = 256;
constexpr int64_t kDeleteChunk = 16384;

WsLayout ws_layout(const svf_params &p, int64_t max_batch);

// Tiered store state (serving form): device cache + host rows + WAVP tables.
struct Tier {
    bool on = false;
    uint8_t *host = nullptr;  // pinned host rows [n_cap][pitch]
    uint8_t *cache = nullptr; // device cache [M][pitch]
    int64_t M = 0;
    int32_t *map = nullptr;   // [n_cap]
    int32_t *owner = nullptr; // [M]
    uint8_t *ref = nullptr;   // [M]
    uint32_t *freq = nullptr; // [n_cap]
    uint32_t *ein = nullptr;  // [n_cap]
    uint32_t *queue = nullptr;
    uint32_t qcap = 0;
    uint64_t *scratch = nullptr;  // maintenance keys
    float alpha = 0.6f, beta = 0.4f, theta = 2.0f, theta0 = 2.0f;
    int promote_batch = 2048, sweep = 4;
    int policy = SVF_TIER_WAVP;
    uint64_t decay_every = 1 << 16;
    int64_t clock = 0;
    uint64_t last_hits = 0, last_misses = 0, misses_at_decay = 0, rounds = 0;
    double last_rate = 0.0, last_meanf = 0.0;
    int64_t M_alloc = 0;           // slots the buffers hold (M <= M_alloc after a reset)
    uint32_t *stat = nullptr;      // [M_alloc][2] LRU / LRFU state
    float lambda = 0.5f;           // LRFU decay per round
    mutable uint32_t tick = 0;     // LRU stamp, advanced per call that reads the tier
};

// Global consolidation in progress (consolidate.cu): a snapshot of the
// graph and deletion bits, the repair's scratch, and the log of the insert
// batches applied to the active graph since the snapshot.
struct LoggedBatch {
    int64_t n0, m, off;  // first new id, rows, offset in the log (rows)
};
struct Consol {
    bool on = false, ran = false, overflow = false;
    int64_t n0 = 0;           // rows in the snapshot
    uint32_t *snap = nullptr; // [n_cap][R]
    uint32_t *snap_del = nullptr;
    uint32_t *vl = nullptr;   // rows to rewrite
    uint32_t *newrows = nullptr;
    uint64_t *cand = nullptr;
    uint32_t *log_rows = nullptr, *log_dkeys = nullptr;  // [log_cap][R]
    unsigned long long *ctr = nullptr;                    // private scan counters
    int64_t log_cap = 0, log_used = 0, rewritten = 0;
    std::vector<LoggedBatch> batches;
    cudaEvent_t done = nullptr;  // end of the run on its stream
};

}  // namespace svf

struct svf_index {
    svf_params p;
    svf_buffers b;
    svf::WsLayout ws;
    int64_t n_used = 0;
    uint64_t repaired = 0;
    int64_t build_fallback = 0;  // rows of the last build whose tensor-core certificate failed
    bool build_tc = false;       // the last build's 2R-NN came from the tensor-core scan
    cudaStream_t last = nullptr;
    svf::Tier tier;
    svf::Consol cons;
    unsigned long long *status() const { return reinterpret_cast<unsigned long long *>(b.status); }
    uint8_t *wsp(size_t off) const { return reinterpret_cast<uint8_t *>(b.workspace) + off; }
    svf::RowDesc prim() const {
        svf::RowDesc r{};
        r.pitch = (int64_t)p.d * svf::esize_of(p.dtype);
        r.base = tier.on ? tier.cache : reinterpret_cast<const uint8_t *>(b.vecs);
        r.map = tier.on ? tier.map : nullptr;
        r.host = tier.on ? tier.host : nullptr;
        r.nchunk = (int)(r.pitch / 16);
        r.d = p.d;
        r.dtype = p.dtype;
        r.metric = p.metric;
        r.copy_bytes = (int)r.pitch;
        svf::set_team(r);
        return r;
    }
    svf::RowDesc lowp(int which) const {
        svf::RowDesc r{};
        r.d = p.d;
        r.metric = p.metric;
        if (which == SVF_BF16) {
            r.base = reinterpret_cast<const uint8_t *>(b.vecs_bf16);
            r.pitch = (int64_t)p.d * 2;
            r.nchunk = p.d / 8;
            r.dtype = SVF_BF16;
            r.copy_bytes = 2 * p.d;
        } else {
            r.base = reinterpret_cast<const uint8_t *>(b.vecs_fp8);
            r.pitch = svf::fp8_pitch(p.d);
            r.nchunk = p.d / 16;
            r.dtype = SVF_FP8;
            r.copy_bytes = (p.d + 4 + 15) / 16 * 16;
        }
        svf::set_team(r);
        return r;
    }
    svf::TierCtx tier_ctx() const {
        svf::TierCtx t{};
        if (!tier.on) return t;
        t.ref = tier.ref;
        t.freq = tier.freq;
        t.ein = tier.ein;
        t.queue = tier.queue;
        t.qcount = status() + svf::kStQCount;
        t.qcap = tier.qcap;
        // what a miss queues: Eq. 2 over theta (WAVP), every miss (CLOCK),
        // F_recent over the fixed theta (LFU), nothing (STATIC)
        t.alpha = tier.policy == SVF_TIER_WAVP ? tier.alpha : 1.f;
        t.beta = tier.policy == SVF_TIER_WAVP ? tier.beta : 0.f;
        const bool lr = tier.policy == SVF_TIER_LRU || tier.policy == SVF_TIER_LRFU;
        t.theta = tier.policy == SVF_TIER_CLOCK || lr ? -1.f
                  : tier.policy == SVF_TIER_STATIC    ? INFINITY
                                                      : tier.theta;
        if (lr) {
            t.stat = tier.stat;
            t.lru = tier.policy == SVF_TIER_LRU;
            t.tick = ++tier.tick;
        }
        return t;
    }
};

namespace svf {
// Global consolidation hooks (consolidate.cu): the insert path logs each
// batch's new rows while a consolidation is in progress; build, attach and
// destroy drop a consolidation in progress.
// Insert / delete with optional version stamping for searches of the
// previous epoch that are still running (serve.cu).  shadow_fits(nvl) tells
// whether the repair's nvl rows fit the update's shadow rows; when it returns
// false the caller has made sure no search of an older epoch is running and
// the rows are rewritten without shadows.
int insert_impl(svf_index *h, const void *X, int64_t m, int32_t L_ins, int32_t T_ins, uint32_t *out_ids,
                cudaStream_t st, const VerUpd *ver);
int delete_impl(svf_index *h, const uint32_t *ids, int64_t m, int64_t *out_newly, cudaStream_t st, const VerUpd *ver,
                const std::function<bool(int64_t)> *shadow_fits);
// Search with an explicit id bound and versioned reads (serve.cu).
int search_at(svf_index *h, const void *Q, int64_t nq, const svf_search_params *sp, uint32_t *out_ids, void *out_dist,
              cudaStream_t st, int64_t n_used, const VerCtx &ver);

cudaError_t consol_log(svf_index *h, int64_t n0, int64_t m, const uint32_t *rows, const uint32_t *dkeys,
                       cudaStream_t st);
void consol_drop(svf_index *h);
}  // namespace svf
