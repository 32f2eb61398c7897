// consolidate.cu -- global consolidation of SVFusion (Sec. 5.2) under the
// multi-version mechanism of Sec. 5.3, on the GPU.
//
// begin:  the graph rows and deletion bits of the moment are copied into a
//         snapshot (caller-provided memory); from then on every insert batch
//         also appends its new rows and their distance keys to a log.
// run:    on the snapshot only (any stream, concurrently with searches and
//         updates of the active graph): every live vertex with at least one
//         deleted out-neighbour is repaired like the localized repair, with
//         every live entry of each deleted neighbour's row as a candidate (at
//         most kMaxRepair in all), reordered by the index's prune.
// commit: (in order with the updates) each logged batch's reverse edges are
//         applied to the consolidated rows of targets inside the snapshot,
//         then those rows replace rows [0, n0) of the active graph; rows
//         inserted since the snapshot are kept as they are (the appended
//         subgraph of Sec. 5.3).
#include <cstring>

#include "index_impl.h"

namespace svf {

namespace {

size_t a256(size_t b) { return (b + 255) / 256 * 256; }


struct ConsLayout {
    size_t snap, snap_del, vl, newrows, cand, log_rows, log_dkeys, ctr, total;
};

ConsLayout cons_layout(const svf_params &p, int64_t log_rows) {
    ConsLayout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += a256(bytes);
        return o;
    };
    const size_t n = (size_t)p.n_cap, R = (size_t)p.R;
    l.snap = take(n * R * 4);
    l.snap_del = take((n + 31) / 32 * 4);
    l.vl = take(n * 4);
    l.newrows = take(n * R * 4);
    l.cand = take((size_t)kDeleteChunk * kMaxRepair * 8);
    l.log_rows = take((size_t)log_rows * R * 4);
    l.log_dkeys = take((size_t)log_rows * R * 4);
    l.ctr = take((size_t)(kStScratch0 + 4) * 8);
    l.total = off;
    return l;
}

}  // namespace

cudaError_t consol_log(svf_index *h, int64_t n0, int64_t m, const uint32_t *rows, const uint32_t *dkeys,
                       cudaStream_t st) {
    Consol &c = h->cons;
    if (!c.on || m == 0) return cudaSuccess;
    if (c.log_used + m > c.log_cap) {
        c.overflow = true;  // commit will refuse; the active graph stays valid
        return cudaSuccess;
    }
    const size_t off = (size_t)c.log_used * h->p.R, bytes = (size_t)m * h->p.R * 4;
    cudaError_t e = cudaMemcpyAsync(c.log_rows + off, rows, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.log_dkeys + off, dkeys, bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    c.batches.push_back({n0, m, c.log_used});
    c.log_used += m;
    return cudaSuccess;
}

void consol_drop(svf_index *h) {
    Consol &c = h->cons;
    if (c.done) {
        cudaEventSynchronize(c.done);  // no run may still write into the caller's buffer
        cudaEventDestroy(c.done);
    }
    c = Consol{};
}

}  // namespace svf

using namespace svf;

extern "C" {

int svf_consolidate_sizes(const svf_params *p, int64_t log_rows, size_t *bytes) {
    if (!p || !bytes) return fail(SVF_EINVAL, "null arguments");
    if (log_rows < 0) return fail(SVF_EINVAL, "log_rows < 0");
    *bytes = cons_layout(*p, log_rows).total;
    return SVF_OK;
}

int svf_consolidate_begin(svf_index *h, void *buf, size_t bytes, int64_t log_rows, void *stream) {
    if (!h || !buf) return fail(SVF_EINVAL, "null index / buffer");
    if (h->cons.on) return fail(SVF_EINVAL, "a consolidation is already in progress (one version at a time)");
    if (h->tier.on) return fail(SVF_EINVAL, "consolidation of a tiered store is not supported");
    if (log_rows < 0) return fail(SVF_EINVAL, "log_rows < 0");
    const ConsLayout l = cons_layout(h->p, log_rows);
    if (bytes < l.total) return fail(SVF_EINVAL, "buffer of %zu bytes, need %zu", bytes, l.total);
    if (reinterpret_cast<uintptr_t>(buf) % 256) return fail(SVF_EINVAL, "buffer must be 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t *b = reinterpret_cast<uint8_t *>(buf);
    Consol c{};
    c.snap = reinterpret_cast<uint32_t *>(b + l.snap);
    c.snap_del = reinterpret_cast<uint32_t *>(b + l.snap_del);
    c.vl = reinterpret_cast<uint32_t *>(b + l.vl);
    c.newrows = reinterpret_cast<uint32_t *>(b + l.newrows);
    c.cand = reinterpret_cast<uint64_t *>(b + l.cand);
    c.log_rows = reinterpret_cast<uint32_t *>(b + l.log_rows);
    c.log_dkeys = reinterpret_cast<uint32_t *>(b + l.log_dkeys);
    c.ctr = reinterpret_cast<unsigned long long *>(b + l.ctr);
    c.n0 = h->n_used;
    c.log_cap = log_rows;
    const int R = h->p.R;
    CUDA_TRY(cudaMemcpyAsync(c.snap, h->b.graph, (size_t)c.n0 * R * 4, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(c.snap_del, h->b.del_bits, (size_t)(h->p.n_cap + 31) / 32 * 4, cudaMemcpyDeviceToDevice,
                             st));
    CUDA_TRY(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming));
    c.on = true;
    h->cons = std::move(c);
    h->last = st;
    return SVF_OK;
}

int svf_consolidate_run(svf_index *h, int32_t cap, int64_t *out_rows, void *stream) {
    if (!h) return fail(SVF_EINVAL, "null index");
    Consol &c = h->cons;
    if (!c.on) return fail(SVF_EINVAL, "no consolidation in progress");
    if (c.ran) return fail(SVF_EINVAL, "the consolidation has already run");
    const int R = h->p.R;
    const RowDesc P = h->prim();
    // default: the most candidates the repair's buffers hold.  (Capping at
    // what the prune can stage in shared memory, 426 rows at d = 96 fp32,
    // measured slower on the 10M x 96 index: 13.8 s against 7.4 s, since a
    // 160 KB staging buffer leaves one prune CTA per SM.)
    if (cap == 0) cap = kMaxRepair;
    if (cap < R || cap > kMaxRepair) return fail(SVF_EINVAL, "cap=%d: need R <= cap <= %d", cap, kMaxRepair);
    cudaStream_t st = (cudaStream_t)stream;
    // rows to rewrite: live rows of the snapshot with a deleted entry
    CUDA_TRY(cudaMemsetAsync(c.ctr, 0, (size_t)(kStScratch0 + 4) * 8, st));
    CUDA_TRY(launch_delete_scan(c.snap, R, c.snap_del, c.n0, 1, c.vl, c.ctr, st));
    unsigned long long nvl = 0;
    CUDA_TRY(cudaMemcpyAsync(&nvl, c.ctr + kStScratch0 + 2, 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t v0 = 0; v0 < (int64_t)nvl; v0 += kDeleteChunk) {
        const int64_t nv = (int64_t)nvl - v0 < kDeleteChunk ? (int64_t)nvl - v0 : kDeleteChunk;
        CUDA_TRY(launch_delete_gather(P, c.snap, R, c.snap_del, c.n0, R, cap, c.vl, v0, nv, c.cand, cap, st));
        PruneArgs a{};
        a.X = P;
        a.cand = c.cand;
        a.cand_stride = cap;
        a.nv = nv;
        a.mode = h->p.prune;
        a.nbr = c.snap;
        a.nbr_w = R;
        a.R = R;
        a.out_rows = c.newrows + v0 * R;
        CUDA_TRY(launch_prune(a, (int)nv, st));
    }
    CUDA_TRY(launch_delete_finalize(c.snap, R, c.snap_del, c.vl, (int64_t)nvl, c.newrows, st));
    CUDA_TRY(cudaEventRecord(c.done, st));
    c.ran = true;
    c.rewritten = (int64_t)nvl;
    if (out_rows) *out_rows = (int64_t)nvl;
    return SVF_OK;
}

int svf_consolidate_commit(svf_index *h, void *stream) {
    if (!h) return fail(SVF_EINVAL, "null index");
    Consol &c = h->cons;
    if (!c.on || !c.ran) return fail(SVF_EINVAL, "no consolidation has run");
    if (c.overflow) {
        consol_drop(h);
        return fail(SVF_ECAPACITY, "the reverse-edge log overflowed; the consolidation was discarded");
    }
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    const int R = h->p.R;
    const RowDesc P = h->prim();
    CUDA_TRY(cudaStreamWaitEvent(st, c.done, 0));
    int32_t *next = reinterpret_cast<int32_t *>(h->wsp(h->ws.region + h->ws.next));
    int32_t *head = reinterpret_cast<int32_t *>(h->wsp(h->ws.head));
    for (const LoggedBatch &lb : c.batches)
        CUDA_TRY(launch_reverse_patch(P, c.snap, R, h->b.del_bits, lb.n0, lb.m, c.log_rows + lb.off * R,
                                      c.log_dkeys + lb.off * R, c.n0, head, next, h->status(), st));
    CUDA_TRY(cudaMemcpyAsync(h->b.graph, c.snap, (size_t)c.n0 * R * 4, cudaMemcpyDeviceToDevice, st));
    h->repaired += (uint64_t)c.rewritten;
    CUDA_TRY(cudaStreamSynchronize(st));
    consol_drop(h);
    return SVF_OK;
}

int svf_consolidate_abort(svf_index *h) {
    if (!h) return fail(SVF_EINVAL, "null index");
    consol_drop(h);
    return SVF_OK;
}

}  // extern "C"
