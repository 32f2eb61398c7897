// api.cu -- the C ABI of include/svf.h: argument validation, workspace
// layout, and the launch sequences of Build / Search / Insert / Delete
// (SVFusion Sec. 2.2, Alg. 1, Sec. 5).  The index borrows every device
// buffer; nothing here allocates device memory.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "index_impl.h"
#include "svf_mlp.h"

using namespace svf;

namespace {
thread_local std::string g_err;
}  // namespace

int svf::fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

WsLayout svf::ws_layout(const svf_params &p, int64_t max_batch) {
    WsLayout w{};
    const int64_t R = p.R, n = p.n_cap;
    size_t off = 0;
    w.head = off;
    off += align256((size_t)n * 4);
    w.vl = off;
    off += align256((size_t)n * 4);
    w.newrows = off;
    off += align256((size_t)n * R * 4);
    w.region = off;
    // build
    size_t b = 0;
    w.knn_keys = b;
    b += align256((size_t)max_batch * 2 * R * 8);
    w.knn_ids = b;
    b += align256((size_t)max_batch * 2 * R * 4);
    w.tc = b;
    w.tc_bytes = tc_build_applies(p.dtype, p.metric, p.d, max_batch, (int)(2 * R))
                     ? tc_build_scratch_bytes(max_batch, p.d, (int)(2 * R))
                     : 0;
    b += align256(w.tc_bytes);
    // insert
    size_t in = 0;
    w.pool = in;
    in += align256((size_t)max_batch * kInsertLmax * 8);
    w.rows = in;
    in += align256((size_t)max_batch * R * 4);
    w.dkeys = in;
    in += align256((size_t)max_batch * R * 4);
    w.next = in;
    in += align256((size_t)max_batch * R * 4);
    // delete
    w.cand = 0;
    size_t de = align256((size_t)kDeleteChunk * kMaxRepair * 8);
    size_t reg = b > in ? b : in;
    reg = reg > de ? reg : de;
    w.total = off + reg;
    w.max_batch = max_batch;
    return w;
}

namespace {
int check_params(const svf_params *p) {
    if (!p) return fail(SVF_EINVAL, "null params");
    if (p->d < 16 || p->d > 2048 || p->d % 16) return fail(SVF_EINVAL, "d=%d: need 16..2048, multiple of 16", p->d);
    if (p->dtype != SVF_F32 && p->dtype != SVF_U8) return fail(SVF_EINVAL, "primary dtype must be F32 or U8");
    if (p->metric != SVF_L2 && p->metric != SVF_IP) return fail(SVF_EINVAL, "bad metric");
    if (p->R != 32 && p->R != 64) return fail(SVF_EINVAL, "R=%d: need 32 or 64", p->R);
    if (p->n_cap < 1 || p->n_cap >= (1LL << 30)) return fail(SVF_EINVAL, "n_cap must be in [1, 2^30)");
    if (p->prune != SVF_PRUNE_RNG && p->prune != SVF_PRUNE_RANK) return fail(SVF_EINVAL, "bad prune mode");
    if (p->repair_c < 1 || p->repair_c * p->R > kMaxRepair)
        return fail(SVF_EINVAL, "repair_c=%d: need 1 <= c and c*R <= %d", p->repair_c, kMaxRepair);
    if (p->lowp && p->dtype != SVF_F32) return fail(SVF_EINVAL, "low-precision copies need an F32 primary store");
    if (p->lowp & ~3) return fail(SVF_EINVAL, "bad lowp bits");
    return SVF_OK;
}
}  // namespace

extern "C" {

const char *svf_last_error(void) { return g_err.c_str(); }

int svf_buffer_sizes(const svf_params *p, int64_t max_batch, svf_sizes *out) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!out || max_batch < 1) return fail(SVF_EINVAL, "bad max_batch / out");
    WsLayout w = ws_layout(*p, max_batch);
    out->vecs = align256((size_t)p->n_cap * p->d * esize_of(p->dtype));
    out->vecs_bf16 = (p->lowp & 1) ? align256((size_t)p->n_cap * p->d * 2) : 0;
    out->vecs_fp8 = (p->lowp & 2) ? align256((size_t)p->n_cap * fp8_pitch(p->d)) : 0;
    out->graph = align256((size_t)p->n_cap * p->R * 4);
    out->del_bits = align256((size_t)((p->n_cap + 31) / 32) * 4);
    out->workspace = w.total;
    out->status = kStWords * 8;
    return SVF_OK;
}

int svf_create(const svf_params *p, const svf_buffers *b, svf_index **out) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!b || !out) return fail(SVF_EINVAL, "null buffers / out");
    if (!b->vecs || !b->graph || !b->del_bits || !b->workspace || !b->status)
        return fail(SVF_EINVAL, "a required device buffer is null");
    if (((p->lowp & 1) && !b->vecs_bf16) || ((p->lowp & 2) && !b->vecs_fp8))
        return fail(SVF_EINVAL, "low-precision store requested but its buffer is null");
    if (b->status_bytes < (size_t)kStWords * 8) return fail(SVF_EINVAL, "status buffer too small");
    // the largest max_batch the workspace supports
    int64_t lo = 0, hi = p->n_cap;
    if (ws_layout(*p, 1).total > b->ws_bytes)
        return fail(SVF_EINVAL, "workspace of %zu bytes is below the minimum %zu", b->ws_bytes, ws_layout(*p, 1).total);
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (ws_layout(*p, mid).total <= b->ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    svf_index *h = new svf_index();
    h->p = *p;
    h->b = *b;
    h->ws = ws_layout(*p, lo);
    cudaError_t e = cudaMemset(b->del_bits, 0, (size_t)((p->n_cap + 31) / 32) * 4);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, (size_t)kStWords * 8);
    if (e == cudaSuccess) e = cudaMemset(b->graph, 0xFF, (size_t)p->n_cap * p->R * 4);
    if (e == cudaSuccess) e = cudaMemset(h->wsp(h->ws.head), 0xFF, (size_t)p->n_cap * 4);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete h;
        return fail(SVF_ECUDA, "initialising buffers: %s", cudaGetErrorString(e));
    }
    *out = h;
    return SVF_OK;
}

int svf_destroy(svf_index *h) {
    if (h) consol_drop(h);
    delete h;
    return SVF_OK;
}

int svf_attach(svf_index *h, int64_t n_used) {
    if (!h) return fail(SVF_EINVAL, "null index");
    if (n_used < 0 || n_used > h->p.n_cap) return fail(SVF_EINVAL, "n_used out of range");
    consol_drop(h);
    h->n_used = n_used;
    return SVF_OK;
}

// Low-precision copies of rows [row0, row0+m); `src` holds those rows
// (device fp32), by default the primary store.
static int encode_lowp(svf_index *h, int64_t row0, int64_t m, cudaStream_t st, const float *src = nullptr) {
    if (!h->p.lowp || m == 0) return SVF_OK;
    if (!src) src = reinterpret_cast<const float *>(h->b.vecs) + row0 * h->p.d;
    if (h->p.lowp & 1)
        CUDA_TRY(launch_encode_bf16(src, m, h->p.d, reinterpret_cast<uint16_t *>(h->b.vecs_bf16) + row0 * h->p.d, st));
    if (h->p.lowp & 2)
        CUDA_TRY(launch_encode_fp8(src, m, h->p.d, reinterpret_cast<uint8_t *>(h->b.vecs_fp8) + row0 * fp8_pitch(h->p.d),
                                   fp8_pitch(h->p.d), st));
    return SVF_OK;
}

int svf_build(svf_index *h, const void *X, int64_t n, void *stream) {
    if (!h || (!X && n > 0)) return fail(SVF_EINVAL, "null index / X");
    if (h->tier.on) return fail(SVF_EINVAL, "build is not available once the store is tiered");
    if (n < 0 || n > h->p.n_cap) return fail(SVF_ECAPACITY, "n=%lld exceeds n_cap", (long long)n);
    if (n > h->ws.max_batch) return fail(SVF_EINVAL, "n=%lld exceeds the workspace's max_batch %lld", (long long)n,
                                         (long long)h->ws.max_batch);
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    consol_drop(h);
    const RowDesc P = h->prim();
    CUDA_TRY(cudaMemcpyAsync(h->b.vecs, X, (size_t)n * P.pitch, cudaMemcpyDeviceToDevice, st));
    int rc = encode_lowp(h, 0, n, st);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(h->b.del_bits, 0, (size_t)((h->p.n_cap + 31) / 32) * 4, st));
    CUDA_TRY(cudaMemsetAsync(h->b.graph, 0xFF, (size_t)h->p.n_cap * h->p.R * 4, st));
    const int K = (int)(n - 1 < 2 * h->p.R ? n - 1 : 2 * h->p.R);
    if (K > 0) {
        uint64_t *keys = reinterpret_cast<uint64_t *>(h->wsp(h->ws.region + h->ws.knn_keys));
        if (K == 2 * h->p.R && h->ws.tc_bytes && tc_build_applies(P.dtype, P.metric, P.d, n, K)) {
            int64_t fb = 0;
            rc = tc_build_knn(P, n, K, reinterpret_cast<uint8_t *>(h->wsp(h->ws.region + h->ws.tc)), h->ws.tc_bytes,
                              keys, &fb, st);
            if (rc) return rc;
            h->build_fallback = fb;
            h->build_tc = true;
        } else {
            CUDA_TRY(launch_knn_self(P, n, 0, n, K, keys, st));
            h->build_fallback = 0;
            h->build_tc = false;
        }
        PruneArgs a{};
        a.X = P;
        a.cand = keys;
        a.cand_stride = K;
        a.nv = n;
        a.mode = h->p.prune;
        a.R = h->p.R;
        a.out_rows = h->b.graph;
        if (h->p.prune == SVF_PRUNE_RANK) {
            uint32_t *ids = reinterpret_cast<uint32_t *>(h->wsp(h->ws.region + h->ws.knn_ids));
            CUDA_TRY(launch_keys_to_out(keys, n, K, K, h->p.dtype, h->p.metric, ids, nullptr, st));
            a.nbr = ids;
            a.nbr_w = K;
        }
        CUDA_TRY(launch_prune(a, (int)(n < (1 << 30) ? n : (1 << 30)), st));
    }
    h->n_used = n;
    return SVF_OK;
}

// Visited-table size (log2 slots) for a pool of L and up to R new ids per
// iteration: never more than half full before a reset; by default the
// smallest power of two >= 4 (L + span * R), and at least 2^10.
static int hash_bits_for(int L, int R, int req, int span = 1) {
    int need = 1;
    while ((1 << need) < 2 * (L + R)) need++;  // table at most half full
    if (req) return req < need ? need : req;
    int b = 1;
    while ((1 << b) < 4 * (L + span * R)) b++;
    return b < 10 ? 10 : b;
}

static int search_impl(svf_index *h, const void *Q, int64_t nq, const svf_search_params *sp, uint32_t *out_ids,
                       void *out_dist, cudaStream_t st, int64_t n_used, const RowDesc &trav,
                       const VerCtx *ver = nullptr) {
    SearchArgs a{};
    if (ver) a.ver = *ver;
    a.trav = trav;
    a.prim = h->prim();
    a.graph = h->b.graph;
    a.del = h->b.del_bits;
    a.n_used = n_used;
    a.Q = Q;
    a.nq = nq;
    a.q_row_bytes = h->p.d * esize_of(h->p.dtype);
    a.q_bytes = (h->p.d * 4 + 15) / 16 * 16;
    a.qkeys = sp->qkeys;
    a.seed = sp->seed ? sp->seed : h->p.seed;
    a.k = sp->k;
    a.T = sp->T;
    a.W = sp->W > 1 ? sp->W : 1;
    // up to W*R new ids per iteration (W parents); with W > 1 the default
    // table holds about four iterations' ids, so resets stay as rare as with
    // one parent per iteration
    a.hash_bits = hash_bits_for(sp->L, a.W * h->p.R, sp->hash_log2, a.W > 1 ? 4 : 1);
    a.rerank = sp->rerank;
    a.out_dtype = h->p.dtype;
    a.out_ids = out_ids;
    a.out_dist = reinterpret_cast<uint32_t *>(out_dist);
    a.pool_out = sp->pool_out;
    a.mlp = sp->mlp;
    a.z_tau = sp->z_tau;
    a.t_min = sp->t_min;
    a.t_every = sp->t_every > 0 ? sp->t_every : 1;
    a.trace_feat = sp->trace_feat;
    a.trace_meta = sp->trace_meta;
    a.status = h->status();
    a.tier = h->tier_ctx();
    CUDA_TRY(launch_search(a, h->p.R, sp->L, st));
    return SVF_OK;
}

// Argument checks of a search; *trav (out) = the store the traversal reads.
static int check_search(svf_index *h, const svf_search_params *sp, RowDesc *trav_out) {
    if (sp->L != 32 && sp->L != 64 && sp->L != 128 && sp->L != 256) return fail(SVF_EINVAL, "L must be 32/64/128/256");
    if (sp->k < 1 || sp->k > 32 || sp->k > sp->L) return fail(SVF_EINVAL, "need 1 <= k <= min(L, 32)");
    if (sp->T < 0) return fail(SVF_EINVAL, "T < 0");
    if (sp->hash_log2 < 0 || sp->hash_log2 > 14) return fail(SVF_EINVAL, "hash_log2 out of range");
    RowDesc trav = h->prim();
    if (sp->precision == SVF_BF16 || sp->precision == SVF_FP8) {
        int bit = sp->precision == SVF_BF16 ? 1 : 2;
        if (!(h->p.lowp & bit)) return fail(SVF_EINVAL, "the index keeps no copy in that precision");
        trav = h->lowp(sp->precision);
    } else if (sp->precision != h->p.dtype) {
        return fail(SVF_EINVAL, "precision must be the primary dtype, SVF_BF16 or SVF_FP8");
    }
    if (sp->rerank && trav.dtype == h->p.dtype) return fail(SVF_EINVAL, "re-rank applies to low-precision traversal");
    if (sp->mlp && sp->t_min < 1) return fail(SVF_EINVAL, "t_min must be >= 1 with a stop network");
    if (sp->W != 0 && sp->W != 1 && sp->W != 2 && sp->W != 4 && sp->W != 8)
        return fail(SVF_EINVAL, "W must be 0, 1, 2, 4 or 8");
    if (sp->W > 1 && (sp->mlp || sp->trace_feat || sp->trace_meta))
        return fail(SVF_EINVAL, "the stop network and traces run with one warp per query (W <= 1)");
    *trav_out = trav;
    return SVF_OK;
}

int svf_search(svf_index *h, const void *Q, int64_t nq, const svf_search_params *sp, uint32_t *out_ids,
               void *out_dist, void *stream) {
    if (!h || !sp) return fail(SVF_EINVAL, "null index / params");
    if (nq < 0) return fail(SVF_EINVAL, "nq < 0");
    if (nq == 0) return SVF_OK;
    if (!Q || !out_ids || !out_dist) return fail(SVF_EINVAL, "null Q / outputs");
    RowDesc trav{};
    if (int rc = check_search(h, sp, &trav)) return rc;
    h->last = (cudaStream_t)stream;
    return search_impl(h, Q, nq, sp, out_ids, out_dist, (cudaStream_t)stream, h->n_used, trav);
}

}  // extern "C"

int svf::search_at(svf_index *h, const void *Q, int64_t nq, const svf_search_params *sp, uint32_t *out_ids,
                   void *out_dist, cudaStream_t st, int64_t n_used, const VerCtx &ver) {
    if (!h || !sp) return fail(SVF_EINVAL, "null index / params");
    if (nq < 0) return fail(SVF_EINVAL, "nq < 0");
    if (nq == 0) return SVF_OK;
    if (!Q || !out_ids || !out_dist) return fail(SVF_EINVAL, "null Q / outputs");
    RowDesc trav{};
    if (int rc = check_search(h, sp, &trav)) return rc;
    if (ver.row_ver && (sp->mlp || sp->trace_feat || sp->trace_meta))
        return fail(SVF_EINVAL, "the stop network and traces are not available to searches that overlap updates");
    return search_impl(h, Q, nq, sp, out_ids, out_dist, st, n_used, trav, &ver);
}

extern "C" {

int svf_insert(svf_index *h, const void *X, int64_t m, int32_t L_ins, int32_t T_ins, uint32_t *out_ids,
               void *stream) {
    return svf::insert_impl(h, X, m, L_ins, T_ins, out_ids, (cudaStream_t)stream, nullptr);
}

}  // extern "C"

int svf::insert_impl(svf_index *h, const void *X, int64_t m, int32_t L_ins, int32_t T_ins, uint32_t *out_ids,
                     cudaStream_t st, const VerUpd *ver) {
    if (!h) return fail(SVF_EINVAL, "null index");
    if (m < 0) return fail(SVF_EINVAL, "m < 0");
    if (m == 0) return SVF_OK;
    if (!X) return fail(SVF_EINVAL, "null X");
    if (h->n_used + m > h->p.n_cap)
        return fail(SVF_ECAPACITY, "n_used %lld + m %lld exceeds n_cap %lld", (long long)h->n_used, (long long)m,
                    (long long)h->p.n_cap);
    if (m > h->ws.max_batch) return fail(SVF_EINVAL, "m exceeds the workspace's max_batch");
    if (L_ins != 32 && L_ins != 64 && L_ins != 128 && L_ins != 256) return fail(SVF_EINVAL, "L_ins must be 32..256");
    if (L_ins < h->p.R) return fail(SVF_EINVAL, "L_ins must be >= R");
    if (T_ins < 0) return fail(SVF_EINVAL, "T_ins < 0");
    if (ver && m * h->p.R > ver->cap) return fail(SVF_ECAPACITY, "insert of %lld rows exceeds the shadow rows", (long long)m);
    h->last = st;
    const RowDesc P = h->prim();
    const int64_t n0 = h->n_used;
    const int R = h->p.R;
    // the new rows: into the primary store (device, or host rows of a tiered
    // store, where they stay uncached until promoted)
    uint8_t *dst = h->tier.on ? h->tier.host : reinterpret_cast<uint8_t *>(h->b.vecs);
    CUDA_TRY(cudaMemcpyAsync(dst + n0 * P.pitch, X, (size_t)m * P.pitch,
                             h->tier.on ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
    int rc = encode_lowp(h, n0, m, st, h->tier.on ? reinterpret_cast<const float *>(X) : nullptr);
    if (rc) return rc;
    uint64_t *pool = reinterpret_cast<uint64_t *>(h->wsp(h->ws.region + h->ws.pool));
    uint32_t *rows = reinterpret_cast<uint32_t *>(h->wsp(h->ws.region + h->ws.rows));
    uint32_t *dkeys = reinterpret_cast<uint32_t *>(h->wsp(h->ws.region + h->ws.dkeys));
    int32_t *next = reinterpret_cast<int32_t *>(h->wsp(h->ws.region + h->ws.next));
    int32_t *head = reinterpret_cast<int32_t *>(h->wsp(h->ws.head));
    // 1. candidate search on the pre-call graph (queries = the new rows)
    svf_search_params sp{};
    sp.k = 1;
    sp.L = L_ins;
    sp.T = T_ins;
    sp.precision = h->p.dtype;
    sp.pool_out = pool;
    rc = search_impl(h, X, m, &sp, rows, dkeys, st, n0, P);
    if (rc) return rc;
    // 2. reorder each pool into the new row
    PruneArgs a{};
    a.X = P;
    a.cand = pool;
    a.cand_stride = L_ins;
    a.nv = m;
    a.mode = h->p.prune;
    a.nbr = h->b.graph;
    a.nbr_w = R;
    a.R = R;
    a.out_rows = rows;
    a.out_dkey = dkeys;
    CUDA_TRY(launch_prune(a, (int)m, st));
    // 3. reverse edges into the tails of the chosen neighbours
    CUDA_TRY(consol_log(h, n0, m, rows, dkeys, st));
    CUDA_TRY(launch_reverse_patch(P, h->b.graph, R, h->b.del_bits, n0, m, rows, dkeys, n0, head, next, h->status(),
                                  st, ver));
    // 4. the new rows
    CUDA_TRY(cudaMemcpyAsync(h->b.graph + n0 * R, rows, (size_t)m * R * 4, cudaMemcpyDeviceToDevice, st));
    if (out_ids) CUDA_TRY(launch_iota(out_ids, m, n0, st));
    h->n_used = n0 + m;
    return SVF_OK;
}

extern "C" {

int svf_delete(svf_index *h, const uint32_t *ids, int64_t m, int64_t *out_newly, void *stream) {
    return svf::delete_impl(h, ids, m, out_newly, (cudaStream_t)stream, nullptr, nullptr);
}

}  // extern "C"

int svf::delete_impl(svf_index *h, const uint32_t *ids, int64_t m, int64_t *out_newly, cudaStream_t st,
                     const VerUpd *ver, const std::function<bool(int64_t)> *shadow_fits) {
    if (!h) return fail(SVF_EINVAL, "null index");
    if (m < 0 || (m > 0 && !ids)) return fail(SVF_EINVAL, "bad ids / m");
    h->last = st;
    unsigned long long *S = h->status();
    const int R = h->p.R;
    CUDA_TRY(cudaMemsetAsync(S + kStScratch0, 0, 4 * 8, st));
    CUDA_TRY(launch_delete_mark(ids, m, h->n_used, h->b.del_bits, S, st, ver));
    uint32_t *vl = reinterpret_cast<uint32_t *>(h->wsp(h->ws.vl));
    CUDA_TRY(launch_delete_scan(h->b.graph, R, h->b.del_bits, h->n_used, R / 2 + 1, vl, S, st));
    unsigned long long hs[3] = {0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(hs, S + kStScratch0, sizeof hs, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hs[0]) return fail(SVF_EINVAL, "delete: id at position %llu is >= n_used; nothing changed", hs[0] - 1);
    if (out_newly) CUDA_TRY(cudaMemcpyAsync(out_newly, S + kStScratch0 + 1, 8, cudaMemcpyDeviceToDevice, st));
    const int64_t nvl = (int64_t)hs[2];
    const RowDesc P = h->prim();
    uint32_t *newrows = reinterpret_cast<uint32_t *>(h->wsp(h->ws.newrows));
    uint64_t *cand = reinterpret_cast<uint64_t *>(h->wsp(h->ws.region + h->ws.cand));
    const int cstride = h->p.repair_c * R;
    for (int64_t v0 = 0; v0 < nvl; v0 += kDeleteChunk) {
        const int64_t nv = nvl - v0 < kDeleteChunk ? nvl - v0 : kDeleteChunk;
        CUDA_TRY(launch_delete_gather(P, h->b.graph, R, h->b.del_bits, h->n_used, h->p.repair_c, kMaxRepair, vl, v0,
                                      nv, cand, cstride, st));
        PruneArgs a{};
        a.X = P;
        a.cand = cand;
        a.cand_stride = cstride;
        a.nv = nv;
        a.mode = h->p.prune;
        a.nbr = h->b.graph;
        a.nbr_w = R;
        a.R = R;
        a.out_rows = newrows + v0 * R;
        CUDA_TRY(launch_prune(a, (int)nv, st));
    }
    // rows read by searches of the previous epoch are shadowed before they
    // are rewritten (unless the caller has none running: too many rows)
    if (ver && nvl > 0 && (!shadow_fits || (*shadow_fits)(nvl)))
        CUDA_TRY(launch_stamp_rows(h->b.graph, R, vl, nvl, *ver, S, st));
    CUDA_TRY(launch_delete_finalize(h->b.graph, R, h->b.del_bits, vl, nvl, newrows, st));
    h->repaired += (uint64_t)nvl;
    return SVF_OK;
}

extern "C" {

int svf_sync(svf_index *h) {
    if (!h) return fail(SVF_EINVAL, "null index");
    CUDA_TRY(cudaStreamSynchronize(h->last));
    unsigned long long e[2] = {0, 0};
    CUDA_TRY(cudaMemcpy(e, h->status(), sizeof e, cudaMemcpyDeviceToHost));
    if (e[0]) {
        unsigned long long z[2] = {0, 0};
        CUDA_TRY(cudaMemcpy(h->status(), z, sizeof z, cudaMemcpyHostToDevice));
        return fail(-(int)e[0], "device-side error %d (detail %llu)", -(int)e[0], e[1]);
    }
    return SVF_OK;
}

int svf_stats(svf_index *h, svf_counters *out) {
    if (!h || !out) return fail(SVF_EINVAL, "null index / out");
    CUDA_TRY(cudaStreamSynchronize(h->last));
    unsigned long long s[kStWords];
    CUDA_TRY(cudaMemcpy(s, h->status(), sizeof s, cudaMemcpyDeviceToHost));
    out->n_used = h->n_used;
    out->n_deleted = (int64_t)s[kStNewlyDeleted];
    out->search_queries = s[kStQueries];
    out->search_iters = s[kStIters];
    out->search_evals = s[kStEvals];
    out->hash_resets = s[kStResets];
    out->repaired_rows = h->repaired;
    out->reverse_targets = s[kStRevTargets];
    out->cache_hits = s[kStHits];
    out->cache_misses = s[kStMisses];
    out->promoted = s[kStPromoted];
    out->evicted = s[kStEvicted];
    out->build_fallback = (uint64_t)h->build_fallback;
    out->build_tensor_core = h->build_tc ? 1u : 0u;
    return SVF_OK;
}

int svf_stats_reset(svf_index *h) {
    if (!h) return fail(SVF_EINVAL, "null index");
    CUDA_TRY(cudaStreamSynchronize(h->last));
    unsigned long long s[kStWords];
    CUDA_TRY(cudaMemcpy(s, h->status(), sizeof s, cudaMemcpyDeviceToHost));
    for (int i = kStQueries; i <= kStRevTargets; i++) s[i] = 0;
    for (int i = kStHits; i <= kStMisses; i++) s[i] = 0;
    s[kStPromoted] = s[kStEvicted] = 0;
    h->tier.last_hits = h->tier.last_misses = h->tier.misses_at_decay = 0;
    h->repaired = 0;
    CUDA_TRY(cudaMemcpy(h->status(), s, sizeof s, cudaMemcpyHostToDevice));
    return SVF_OK;
}

int svf_encode_bf16(const float *X, int64_t n, int32_t d, void *out, void *stream) {
    if (n < 0 || d <= 0 || (n > 0 && (!X || !out))) return fail(SVF_EINVAL, "bad arguments");
    CUDA_TRY(launch_encode_bf16(X, n, d, reinterpret_cast<uint16_t *>(out), (cudaStream_t)stream));
    return SVF_OK;
}

int svf_encode_fp8(const float *X, int64_t n, int32_t d, void *out, int64_t pitch, void *stream) {
    if (n < 0 || d <= 0 || pitch < d + 4 || pitch % 16 || (n > 0 && (!X || !out))) return fail(SVF_EINVAL, "bad arguments");
    CUDA_TRY(launch_encode_fp8(X, n, d, reinterpret_cast<uint8_t *>(out), pitch, (cudaStream_t)stream));
    return SVF_OK;
}

int svf_knn(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t metric, const void *Q, int64_t nq,
            const int64_t *self, int32_t k, uint64_t *work_keys, uint32_t *out_ids, void *out_dist, void *stream) {
    if (n < 1 || nq < 0 || d < 16 || d > 2048 || d % 16 || k < 1 || k > 128)
        return fail(SVF_EINVAL, "bad sizes (n >= 1, d multiple of 16 in 16..2048, 1 <= k <= 128)");
    if (dtype != SVF_F32 && dtype != SVF_U8) return fail(SVF_EINVAL, "dtype must be F32 or U8");
    if (metric != SVF_L2 && metric != SVF_IP) return fail(SVF_EINVAL, "bad metric");
    if (nq == 0) return SVF_OK;
    if (!X || !Q || !work_keys || !out_ids) return fail(SVF_EINVAL, "null pointers");
    cudaStream_t st = (cudaStream_t)stream;
    KnnArgs a{};
    a.X.base = reinterpret_cast<const uint8_t *>(X);
    a.X.pitch = (int64_t)d * esize_of(dtype);
    a.X.nchunk = (int)(a.X.pitch / 16);
    a.X.d = d;
    a.X.dtype = dtype;
    a.X.metric = metric;
    a.X.copy_bytes = (int)a.X.pitch;
    set_team(a.X);
    a.n = n;
    a.Q = Q;
    a.q_row_bytes = (int)a.X.pitch;
    a.nq = nq;
    a.self = self;
    a.self_base = -1;
    a.k = k;
    a.out_keys = work_keys;
    CUDA_TRY(launch_knn(a, st));
    CUDA_TRY(launch_keys_to_out(work_keys, nq, k, k, dtype, metric, out_ids, reinterpret_cast<uint32_t *>(out_dist), st));
    return SVF_OK;
}

int svf_mlp_grad(const float *feat, const int32_t *meta, int32_t T, const int32_t *idx, int64_t B, const float *params,
                 float *grad, float *partial, float *loss, void *stream) {
    if (!feat || !meta || !idx || !params || !grad || !partial || B < 1 || T < 1)
        return fail(SVF_EINVAL, "bad arguments");
    CUDA_TRY(launch_mlp_grad(feat, meta, T, idx, B, params, grad, partial, loss, (cudaStream_t)stream));
    return SVF_OK;
}

int64_t svf_mlp_partial_floats(int64_t B) { return B < 1 ? 0 : (int64_t)mlp_grad_partial_floats(B); }

int svf_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t step, float lr, float beta1,
                 float beta2, float eps, void *stream) {
    if (!params || !grad || !m || !v || step < 1) return fail(SVF_EINVAL, "bad arguments");
    CUDA_TRY(launch_mlp_adam(params, grad, m, v, step, lr, beta1, beta2, eps, (cudaStream_t)stream));
    return SVF_OK;
}

int svf_mlp_pack(const float *params, void *packed, void *stream) {
    if (!params || !packed) return fail(SVF_EINVAL, "bad arguments");
    CUDA_TRY(launch_mlp_pack(params, packed, (cudaStream_t)stream));
    return SVF_OK;
}

int svf_mlp_forward(const float *params, const float *feat, int64_t n, float *z, void *stream) {
    if (n < 0 || (n > 0 && (!params || !feat || !z))) return fail(SVF_EINVAL, "bad arguments");
    CUDA_TRY(launch_mlp_forward(params, feat, n, z, (cudaStream_t)stream));
    return SVF_OK;
}

}  // extern "C"
