// serve.cu -- continuous-batching request loop over one index (SVFusion's
// real-time coordination, Sec. 4.4, and consistency, Sec. 5.3).
//
// A worker thread admits requests in arrival order.  Search batches are
// launched on a pool of streams as soon as they arrive and fewer than
// max_inflight batches are on the GPU, so batches of uneven size overlap on
// the device.  An insert or delete is an epoch boundary: admission pauses,
// the in-flight searches finish, the update runs alone on its stream, the
// epoch advances, and later searches see the new state.  Every search
// therefore reads exactly the index state of its epoch, and its result
// equals a run of the same search alone on that state.  Tier maintenance
// (promotion / eviction, Alg. 2) also runs only between epochs' searches.
// Host timestamps (steady clock) give per-request latency.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "index_impl.h"

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

    void run() {
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

int svf_serve_start(svf_index *h, const svf_serve_cfg *cfg, svf_server **out) {
    if (!h || !cfg || !out) return svf::fail(SVF_EINVAL, "null arguments");
    if (cfg->max_inflight < 1 || cfg->n_streams < 1 || cfg->n_streams > 64)
        return svf::fail(SVF_EINVAL, "need max_inflight >= 1 and 1 <= n_streams <= 64");
    svf_server *s = new svf_server();
    s->h = h;
    s->cfg = *cfg;
    if (s->cfg.maintain_every < 1) s->cfg.maintain_every = 64;
    cudaGetDevice(&s->device);
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
    delete s;
    return SVF_OK;
}

}  // extern "C"
