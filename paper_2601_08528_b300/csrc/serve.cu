// serve.cu -- continuous-batching request loop over one index (SVFusion's
// real-time coordination, Sec. 4.4, and consistency, Sec. 5.3).
//
// A worker thread admits requests in arrival order.  Search batches are
// launched on a pool of streams as soon as they arrive and fewer than
// max_inflight batches are on the GPU, so batches of uneven size overlap on
// the device.  Inserts and deletes run one at a time on a dedicated update
// stream.  In the barrier mode an update waits for the in-flight searches
// and later searches wait for it.  In the versioned modes an update runs
// while the searches admitted before it are still on the GPU: it stamps and
// shadows every existing row it rewrites and every vertex it deletes, and a
// search reads the graph as of its epoch (VerCtx).  Read-after-write: a
// search's epoch counts every update submitted before it and its stream waits
// for the last of them.  Snapshot: a search's epoch counts the updates that
// had completed when it was admitted, and it waits for none.  Update E + 1
// starts only when no search of an epoch below E is running, so each row
// needs one shadow.  Every search therefore reads exactly the index state of
// its epoch, and its result equals a run of the same search alone on that
// state.  Tier maintenance (promotion / eviction, Alg. 2) runs only while no
// search or update is in flight.  Host timestamps (steady clock) give
// per-request latency.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "index_impl.h"
#include "svf_update.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Inflight {
    svf_request req;
    cudaEvent_t ev;
    double t_start;
    uint64_t epoch;
};

// An update launched on the update stream, not yet known complete.
struct UpdFlight {
    svf_request req;
    cudaEvent_t ev;
    uint64_t E;
    int64_t n_after;   // n_used once it completes
    double t_start;
    int rc;
    bool barrier;      // ran with no older search in flight; later searches wait for it
};

// Version buffer layout (256-byte aligned pieces).
struct VerLayout {
    size_t row_ver, shadow_slot, del_ep, counter, shadow, total;
};
VerLayout ver_layout(int64_t n_cap, int R, int64_t shadow_rows) {
    VerLayout L{};
    size_t o = 0;
    auto take = [&](size_t b) {
        size_t at = o;
        o += svf::align256(b);
        return at;
    };
    L.row_ver = take((size_t)n_cap * 4);
    L.shadow_slot = take((size_t)n_cap * 4);
    L.del_ep = take((size_t)n_cap * 4);
    L.counter = take(256);
    L.shadow = take((size_t)2 * shadow_rows * R * 4);
    L.total = o;
    return L;
}

// del_ep of a vertex already deleted when serving starts: 0 (every epoch sees it deleted)
__global__ void init_del_ep_kernel(const uint32_t *del, int64_t n_cap, uint32_t *del_ep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_cap) del_ep[i] = ((del[i >> 5] >> (i & 31)) & 1u) ? 0u : 0xFFFFFFFFu;
}

}  // namespace

struct svf_server {
    svf_index *h = nullptr;
    svf_serve_cfg cfg{};
    std::vector<cudaStream_t> streams;
    cudaStream_t upd = nullptr;
    std::vector<cudaEvent_t> free_ev;
    cudaEvent_t upd_ev = nullptr;
    bool have_upd_ev = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<svf_request> queue;
    std::deque<svf_completion> done;
    std::vector<Inflight> inflight;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<uint64_t> submitted{0}, completed{0};
    uint64_t epoch = 0;
    int rr = 0;
    int since_maint = 0;
    int device = 0;
    int first_error = 0;
    // versioned modes
    uint32_t *row_ver = nullptr, *del_ep = nullptr, *shadow = nullptr;
    int32_t *shadow_slot = nullptr;
    unsigned long long *counter = nullptr;
    uint64_t committed = 0, launched = 0;  // updates completed / launched
    int64_t n_committed = 0;               // n_used after the completed updates
    std::deque<svf_request> upd_q;         // updates accepted, not launched
    std::deque<UpdFlight> upd_fl;          // updates launched, not known complete
    cudaEvent_t commit_ev = nullptr;       // the last completed update (memory order for new searches)
    bool have_commit_ev = false;

    void complete(const svf_request &r, int status, uint64_t ep, double t0, double t1) {
        svf_completion c{};
        c.tag = r.tag;
        c.op = r.op;
        c.status = status;
        c.epoch = ep;
        c.count = r.count;
        c.t_arrival = r.t_arrival;
        c.t_start = t0;
        c.t_done = t1;
        {
            std::lock_guard<std::mutex> lk(mu);
            done.push_back(c);
        }
        if (status && !first_error) first_error = status;
        completed++;
    }

    void reap(bool all) {
        do {
            for (size_t i = 0; i < inflight.size();) {
                cudaError_t q = cudaEventQuery(inflight[i].ev);
                if (q == cudaErrorNotReady) {
                    i++;
                    continue;
                }
                const double t = now_s();
                complete(inflight[i].req, q == cudaSuccess ? SVF_OK : SVF_ECUDA, inflight[i].epoch, inflight[i].t_start, t);
                free_ev.push_back(inflight[i].ev);
                inflight[i] = inflight.back();
                inflight.pop_back();
            }
            if (all && !inflight.empty()) std::this_thread::yield();
        } while (all && !inflight.empty());
    }

    void maintain_if_due() {
        if (!h->tier.on || since_maint < cfg.maintain_every) return;
        reap(true);
        int64_t np = 0;
        svf_tier_maintain(h, &np, upd);
        cudaStreamSynchronize(upd);
        since_maint = 0;
    }

    svf::VerCtx ver_ctx(uint64_t e) const {
        svf::VerCtx v{};
        v.row_ver = row_ver;
        v.shadow_slot = shadow_slot;
        v.shadow = shadow;
        v.del_ep = del_ep;
        v.epoch = (uint32_t)e;
        return v;
    }

    cudaEvent_t take_event() {
        cudaEvent_t ev;
        if (free_ev.empty()) {
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        } else {
            ev = free_ev.back();
            free_ev.pop_back();
        }
        return ev;
    }

    // Updates whose work has completed, in order.
    void poll_updates() {
        while (!upd_fl.empty() && cudaEventQuery(upd_fl.front().ev) != cudaErrorNotReady) {
            UpdFlight &u = upd_fl.front();
            committed = u.E;
            n_committed = u.n_after;
            if (have_commit_ev) free_ev.push_back(commit_ev);
            commit_ev = u.ev;
            have_commit_ev = true;
            complete(u.req, u.rc, u.E, u.t_start, now_s());
            upd_fl.pop_front();
        }
    }

    bool old_search_running(uint64_t below) const {
        for (const auto &f : inflight)
            if (f.epoch < below) return true;
        return false;
    }

    // Launch the next accepted update when the previous one has completed and
    // no search older than it is still reading its shadows.
    void try_launch_update() {
        if (upd_q.empty() || !upd_fl.empty() || old_search_running(committed)) return;
        if (h->tier.on && since_maint >= cfg.maintain_every) return;  // maintenance first
        svf_request r = upd_q.front();
        upd_q.pop_front();
        const uint64_t E = launched + 1;
        svf::VerUpd v{};
        v.E = (uint32_t)E;
        v.row_ver = row_ver;
        v.shadow_slot = shadow_slot;
        v.shadow = shadow;
        v.base = (E & 1) ? cfg.shadow_rows : 0;
        v.cap = cfg.shadow_rows;
        v.del_ep = del_ep;
        v.counter = counter;
        bool barrier = false;
        const double t0 = now_s();
        int rc = SVF_EINVAL;
        cudaMemsetAsync(counter, 0, 8, upd);
        if (r.op == SVF_OP_INSERT) {
            if ((int64_t)r.count * h->p.R > cfg.shadow_rows) {
                reap(true);  // too many rows to shadow: run with no older search in flight
                barrier = true;
                rc = svf::insert_impl(h, r.data, r.count, r.L_ins, r.T_ins, r.out_new_ids, upd, nullptr);
            } else {
                rc = svf::insert_impl(h, r.data, r.count, r.L_ins, r.T_ins, r.out_new_ids, upd, &v);
            }
        } else if (r.op == SVF_OP_DELETE) {
            std::function<bool(int64_t)> fits = [&](int64_t nvl) {
                if (nvl <= cfg.shadow_rows) return true;
                reap(true);
                barrier = true;
                return false;
            };
            rc = svf::delete_impl(h, reinterpret_cast<const uint32_t *>(r.data), r.count, nullptr, upd, &v, &fits);
        }
        cudaEvent_t ev = take_event();
        cudaEventRecord(ev, upd);
        upd_fl.push_back({r, ev, E, h->n_used, t0, rc, barrier});
        launched = E;
    }

    void maintain_versioned() {
        if (!h->tier.on || since_maint < cfg.maintain_every) return;
        reap(true);
        cudaStreamSynchronize(upd);
        poll_updates();
        int64_t np = 0;
        svf_tier_maintain(h, &np, upd);
        cudaStreamSynchronize(upd);
        since_maint = 0;
    }

    void run_versioned() {
        cudaSetDevice(device);
        n_committed = h->n_used;
        const bool snapshot = cfg.consistency == SVF_SERVE_SNAPSHOT;
        while (true) {
            reap(false);
            poll_updates();
            try_launch_update();
            svf_request r;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (queue.empty()) {
                    if (stop && inflight.empty() && upd_q.empty() && upd_fl.empty()) return;
                    lk.unlock();
                    if (inflight.empty() && upd_fl.empty() && since_maint > 0 && h->tier.on) maintain_versioned();
                    std::this_thread::yield();
                    continue;
                }
                r = queue.front();
            }
            if (r.t_arrival > 0 && now_s() < r.t_arrival) {
                std::this_thread::yield();
                continue;
            }
            if (r.op != SVF_OP_SEARCH) {
                {
                    std::lock_guard<std::mutex> lk(mu);
                    queue.pop_front();
                }
                upd_q.push_back(r);
                continue;
            }
            if ((int)inflight.size() >= cfg.max_inflight) continue;
            if (h->tier.on && since_maint >= cfg.maintain_every) {
                maintain_versioned();
                continue;
            }
            // the epoch this search reads, its id bound, and the update it waits for
            uint64_t e;
            int64_t n;
            cudaEvent_t wait = nullptr;
            const bool barrier_fl = !upd_fl.empty() && upd_fl.back().barrier;
            if (!snapshot || barrier_fl) {
                if (!upd_q.empty()) continue;  // it must see an update not launched yet
                e = launched;
                n = h->n_used;
                if (!upd_fl.empty()) wait = upd_fl.back().ev;
                else if (have_commit_ev) wait = commit_ev;
            } else {
                e = committed;
                n = n_committed;
                if (have_commit_ev) wait = commit_ev;
            }
            cudaStream_t s = streams[rr++ % streams.size()];
            if (wait) cudaStreamWaitEvent(s, wait, 0);
            cudaEvent_t ev = take_event();
            const double t0 = now_s();
            int rc = svf::search_at(h, r.data, r.count, &r.sp, r.out_ids, r.out_dist, s, n, ver_ctx(e));
            {
                std::lock_guard<std::mutex> lk(mu);
                queue.pop_front();
            }
            if (rc) {
                complete(r, rc, e, t0, now_s());
                free_ev.push_back(ev);
                continue;
            }
            cudaEventRecord(ev, s);
            inflight.push_back({r, ev, t0, e});
            since_maint++;
        }
    }

    void run() {
        if (cfg.consistency != SVF_SERVE_BARRIER) return run_versioned();
        cudaSetDevice(device);
        while (true) {
            reap(false);
            svf_request r;
            {
                std::unique_lock<std::mutex> lk(mu);
                if (queue.empty()) {
                    if (stop && inflight.empty()) return;
                    lk.unlock();
                    if (inflight.empty() && since_maint > 0 && h->tier.on) maintain_if_due();
                    std::this_thread::yield();
                    continue;
                }
                r = queue.front();
            }
            // open-loop replay: a request starts no earlier than its arrival
            if (r.t_arrival > 0 && now_s() < r.t_arrival) {
                std::this_thread::yield();
                continue;
            }
            if (r.op == SVF_OP_SEARCH) {
                if ((int)inflight.size() >= cfg.max_inflight) continue;
                if (h->tier.on && since_maint >= cfg.maintain_every) {
                    maintain_if_due();
                    continue;
                }
                cudaStream_t s = streams[rr++ % streams.size()];
                if (have_upd_ev) cudaStreamWaitEvent(s, upd_ev, 0);
                cudaEvent_t ev;
                if (free_ev.empty()) {
                    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                } else {
                    ev = free_ev.back();
                    free_ev.pop_back();
                }
                const double t0 = now_s();
                int rc = svf_search(h, r.data, r.count, &r.sp, r.out_ids, r.out_dist, s);
                {
                    std::lock_guard<std::mutex> lk(mu);
                    queue.pop_front();
                }
                if (rc) {
                    complete(r, rc, epoch, t0, now_s());
                    free_ev.push_back(ev);
                    continue;
                }
                cudaEventRecord(ev, s);
                inflight.push_back({r, ev, t0, epoch});
                since_maint++;
            } else {
                // epoch boundary: the update runs alone
                reap(true);
                maintain_if_due();
                const double t0 = now_s();
                int rc = SVF_EINVAL;
                if (r.op == SVF_OP_INSERT)
                    rc = svf_insert(h, r.data, r.count, r.L_ins, r.T_ins, r.out_new_ids, upd);
                else if (r.op == SVF_OP_DELETE)
                    rc = svf_delete(h, reinterpret_cast<const uint32_t *>(r.data), r.count, nullptr, upd);
                cudaEventRecord(upd_ev, upd);
                have_upd_ev = true;
                cudaStreamSynchronize(upd);
                {
                    std::lock_guard<std::mutex> lk(mu);
                    queue.pop_front();
                }
                epoch++;
                complete(r, rc, epoch, t0, now_s());
            }
        }
    }
};

extern "C" {

double svf_serve_now(void) { return now_s(); }

size_t svf_serve_version_bytes(svf_index *h, int64_t shadow_rows) {
    if (!h || shadow_rows < 1) return 0;
    return ver_layout(h->p.n_cap, h->p.R, shadow_rows).total;
}

int svf_serve_start(svf_index *h, const svf_serve_cfg *cfg, svf_server **out) {
    if (!h || !cfg || !out) return svf::fail(SVF_EINVAL, "null arguments");
    if (cfg->max_inflight < 1 || cfg->n_streams < 1 || cfg->n_streams > 64)
        return svf::fail(SVF_EINVAL, "need max_inflight >= 1 and 1 <= n_streams <= 64");
    if (cfg->consistency < SVF_SERVE_BARRIER || cfg->consistency > SVF_SERVE_SNAPSHOT)
        return svf::fail(SVF_EINVAL, "bad consistency mode");
    VerLayout VL{};
    if (cfg->consistency != SVF_SERVE_BARRIER) {
        if (cfg->shadow_rows < 1 || cfg->shadow_rows >= (1ll << 30))
            return svf::fail(SVF_EINVAL, "shadow_rows must be in [1, 2^30)");
        VL = ver_layout(h->p.n_cap, h->p.R, cfg->shadow_rows);
        if (!cfg->versions || cfg->versions_bytes < VL.total)
            return svf::fail(SVF_EINVAL, "version buffer of %zu bytes, need %zu", cfg->versions_bytes, VL.total);
    }
    svf_server *s = new svf_server();
    s->h = h;
    s->cfg = *cfg;
    if (s->cfg.maintain_every < 1) s->cfg.maintain_every = 64;
    cudaGetDevice(&s->device);
    if (cfg->consistency != SVF_SERVE_BARRIER) {
        uint8_t *B = reinterpret_cast<uint8_t *>(cfg->versions);
        s->row_ver = reinterpret_cast<uint32_t *>(B + VL.row_ver);
        s->shadow_slot = reinterpret_cast<int32_t *>(B + VL.shadow_slot);
        s->del_ep = reinterpret_cast<uint32_t *>(B + VL.del_ep);
        s->counter = reinterpret_cast<unsigned long long *>(B + VL.counter);
        s->shadow = reinterpret_cast<uint32_t *>(B + VL.shadow);
        const int64_t nc = h->p.n_cap;
        // the index's own stream work (earlier calls) comes first
        if (h->last) cudaStreamSynchronize(h->last);
        cudaMemset(s->row_ver, 0, (size_t)nc * 4);
        cudaMemset(s->shadow_slot, 0xFF, (size_t)nc * 4);
        cudaMemset(s->counter, 0, 8);
        init_del_ep_kernel<<<(unsigned)((nc + 255) / 256), 256>>>(h->b.del_bits, nc, s->del_ep);
        if (cudaDeviceSynchronize() != cudaSuccess) {
            delete s;
            return svf::fail(SVF_ECUDA, "version buffer initialisation failed");
        }
    }
    for (int i = 0; i < cfg->n_streams; i++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return svf::fail(SVF_ECUDA, "stream creation failed");
        }
        s->streams.push_back(st);
    }
    cudaStreamCreateWithFlags(&s->upd, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s->upd_ev, cudaEventDisableTiming);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return SVF_OK;
}

int svf_serve_submit(svf_server *s, const svf_request *r) {
    if (!s || !r) return svf::fail(SVF_EINVAL, "null arguments");
    if (r->op != SVF_OP_SEARCH && r->op != SVF_OP_INSERT && r->op != SVF_OP_DELETE)
        return svf::fail(SVF_EINVAL, "bad op");
    if (s->stop) return svf::fail(SVF_EINVAL, "server is stopping");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.push_back(*r);
    }
    s->submitted++;
    return SVF_OK;
}

int svf_serve_poll(svf_server *s, svf_completion *out, int max, int *n_out) {
    if (!s || (!out && max > 0) || !n_out) return svf::fail(SVF_EINVAL, "null arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    return SVF_OK;
}

int svf_serve_drain(svf_server *s, double timeout_s) {
    if (!s) return svf::fail(SVF_EINVAL, "null server");
    const double t_end = now_s() + timeout_s;
    while (s->completed.load() < s->submitted.load()) {
        if (now_s() > t_end) return svf::fail(SVF_ETIMEOUT, "drain timed out");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return s->first_error;
}

int svf_serve_stop(svf_server *s) {
    if (!s) return svf::fail(SVF_EINVAL, "null server");
    s->stop = true;
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->streams) cudaStreamSynchronize(st);
    cudaStreamSynchronize(s->upd);
    s->h->last = nullptr;  // the index's calls went to the server's streams
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (auto ev : s->free_ev) cudaEventDestroy(ev);
    cudaStreamDestroy(s->upd);
    cudaEventDestroy(s->upd_ev);
    if (s->have_commit_ev) cudaEventDestroy(s->commit_ev);
    delete s;
    return SVF_OK;
}

}  // extern "C"
