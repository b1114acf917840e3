// Request server: continuous batching of blockBP solves on one GPU.
//
// Requests (a lattice description, its tensors and the observables to read) are queued
// by bbp_server_submit.  A worker thread admits queued requests in arrival order as
// soon as their planned device footprint fits in the server's byte budget (and a slot
// is free), uploads them, and keeps one sweep of every admitted solve in flight, each
// on the solve's own stream, so that the kernels of different solves overlap on the
// device.  A solve whose residual meets its tolerance (or that reaches max_sweeps) is
// handed to a second thread that reads it out (bbp_expect) and releases it, so that the
// sweeps of the other solves keep flowing meanwhile; its bytes then go to the next
// admissions.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bbp.h"
#include "engine.h"
#include "lattice.h"

using namespace bbp;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct TermCopy {
    int nsite = 1;
    int site[2] = {0, 0};
    std::vector<double> re[2], im[2];
    bool has_im[2] = {false, false};
};

struct Request {
    long long id = 0;
    bbp_lattice_desc desc{};
    std::vector<unsigned char> tensors;
    std::vector<TermCopy> terms;
    size_t footprint = 0;
    int state = 0;  // 0 queued, 1 running, 2 done, < 0 error code
    bbp_lattice* L = nullptr;
    bool in_flight = false;
    int sweeps = 0;
    double residual = 0.0;
    std::vector<double> out_re, out_im;
    double t_submit = 0, t_admit = 0, t_finish = 0;
    std::string error;
};

}  // namespace

struct bbp_server {
    size_t max_bytes = 0;
    int max_active = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<long long, std::unique_ptr<Request>> reqs;
    std::vector<Request*> active;  // worker thread only
    std::deque<Request*> ro_queue;  // converged solves waiting for their read-out
    std::condition_variable cv_ro;
    size_t used = 0;
    long long next_id = 1;
    std::atomic<bool> stop{false};
    bool ro_stop = false;
    std::thread worker, ro_worker;
    std::atomic<long long> sweeps_total{0};

    void run();
    void run_readouts();
    int readout(Request* r);
    void finish(Request* r, int rc, const std::string& err);
};

int bbp_server::readout(Request* r) {
    const int n = (int)r->terms.size();
    std::vector<bbp_term> ts(n);
    for (int k = 0; k < n; ++k) {
        ts[k].nsite = r->terms[k].nsite;
        for (int j = 0; j < r->terms[k].nsite; ++j) {
            ts[k].site[j] = r->terms[k].site[j];
            ts[k].op_re[j] = r->terms[k].re[j].data();
            ts[k].op_im[j] = r->terms[k].has_im[j] ? r->terms[k].im[j].data() : nullptr;
        }
    }
    r->out_re.assign(n, 0.0);
    r->out_im.assign(n, 0.0);
    return n ? bbp_expect(r->L, ts.data(), n, r->out_re.data(), r->out_im.data()) : BBP_OK;
}

void bbp_server::run_readouts() {
    cudaSetDevice(device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_ro.wait(lk, [this] { return !ro_queue.empty() || ro_stop; });
            if (ro_queue.empty()) return;  // stopping and drained
            r = ro_queue.front();
            ro_queue.pop_front();
        }
        const int rc = readout(r);
        finish(r, rc, rc ? bbp_last_error() : "");
    }
}

void bbp_server::finish(Request* r, int rc, const std::string& err) {
    if (r->L) {
        bbp_destroy(r->L);
        r->L = nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    used -= r->footprint;
    r->state = rc < 0 ? rc : 2;
    r->error = err;
    r->t_finish = now_s();
    cv_done.notify_all();
}

void bbp_server::run() {
    cudaSetDevice(device);
    for (;;) {
        // admission by footprint, in arrival order (a request that does not fit yet
        // does not block smaller ones behind it)
        std::vector<Request*> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty() && queue.empty()) {
                if (stop) return;
                cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            for (auto it = queue.begin(); it != queue.end();) {
                Request* r = *it;
                if ((int)(active.size() + admit.size()) < max_active && used + r->footprint <= max_bytes) {
                    used += r->footprint;
                    admit.push_back(r);
                    it = queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        for (Request* r : admit) {
            r->t_admit = now_s();
            bbp_lattice_desc d = r->desc;
            d.stream = nullptr;  // every solve gets its own stream
            int rc = bbp_create_lattice(&d, &r->L);
            if (!rc) rc = bbp_set_tensors(r->L, r->tensors.data(), 0);
            if (rc) {
                finish(r, rc, bbp_last_error());
                continue;
            }
            {
                std::lock_guard<std::mutex> g(mu);
                r->state = 1;
            }
            active.push_back(r);
        }
        bool progressed = !admit.empty();
        for (size_t i = 0; i < active.size();) {
            Request* r = active[i];
            bool done = false;
            int rc = 0;
            if (r->L->items.empty()) {  // one block covering everything: read out directly
                done = true;
            } else if (!r->in_flight) {
                rc = sweep_launch(r->L);
                r->in_flight = rc == 0;
                progressed = true;
            } else if (sweep_ready(r->L)) {
                bool conv = false;
                rc = sweep_collect(r->L, &r->residual, &conv);
                r->in_flight = false;
                progressed = true;
                if (!rc) {
                    r->sweeps++;
                    sweeps_total++;
                    done = conv || r->sweeps >= std::max(1, r->desc.max_sweeps);
                    if (!done) {
                        rc = sweep_launch(r->L);
                        r->in_flight = rc == 0;
                    }
                }
            }
            if (!rc && done) {  // converged: the read-out thread takes the solve from here
                {
                    std::lock_guard<std::mutex> g(mu);
                    ro_queue.push_back(r);
                }
                cv_ro.notify_one();
                active.erase(active.begin() + i);
                progressed = true;
            } else if (rc) {
                finish(r, rc, bbp_last_error());
                active.erase(active.begin() + i);
                progressed = true;
            } else {
                ++i;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Entries of a term's operator at `site`: d x d, or on a single-layer network the impurity
// tensor with the site tensor's shape (OBC edge legs of dimension 1); 0 for a site outside
// the lattice (OBC) or the block (INFINITE).
static size_t op_entries(const bbp_lattice_desc& ds, int site) {
    if (!ds.single_layer) return (size_t)ds.d * ds.d;
    const bool obc = ds.boundary == BBP_OBC;
    const int W = obc ? ds.Lx : ds.bx, H = obc ? ds.Ly : ds.by, D = ds.D;
    if (site < 0 || site >= W * H) return 0;
    if (!obc) return (size_t)D * D * D * D;
    const int r = site / W, c = site % W;
    return (size_t)(r == 0 ? 1 : D) * (c == 0 ? 1 : D) * (r == H - 1 ? 1 : D) * (c == W - 1 ? 1 : D);
}

extern "C" {

int bbp_server_create(size_t max_bytes, int max_active, bbp_server** out) try {
    if (!out || max_bytes == 0 || max_active < 1) return fail(BBP_ERR_INVALID, "server: need out, max_bytes > 0, max_active >= 1");
    bbp_server* s = new (std::nothrow) bbp_server();
    if (!s) return fail(BBP_ERR_OOM, "server: host allocation failed");
    s->max_bytes = max_bytes;
    s->max_active = max_active;
    if (cudaGetDevice(&s->device) != cudaSuccess) s->device = 0;
    try {
        s->worker = std::thread([s] { s->run(); });
        s->ro_worker = std::thread([s] { s->run_readouts(); });
    } catch (...) {
        // a thread could not start: stop the one that did, then report
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stop = true;
            s->ro_stop = true;
        }
        s->cv_work.notify_all();
        s->cv_ro.notify_all();
        if (s->worker.joinable()) s->worker.join();
        if (s->ro_worker.joinable()) s->ro_worker.join();
        delete s;
        return fail(BBP_ERR_OOM, "server: a worker thread could not start");
    }
    *out = s;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_server_submit(bbp_server* s, const bbp_lattice_desc* desc, const void* tensors, const bbp_term* terms,
                      int n_terms, long long* id) try {
    if (!s || !desc || !tensors || !id || n_terms < 0 || (n_terms > 0 && !terms))
        return fail(BBP_ERR_INVALID, "server_submit: bad arguments");
    bbp_lattice* plan = nullptr;
    int rc = plan_lattice(desc, &plan);
    if (rc) return rc;
    auto r = std::make_unique<Request>();
    r->desc = *desc;
    r->footprint = planned_bytes(plan);
    const size_t raw_bytes = plan->raw_bytes;
    delete plan;
    if (r->footprint > s->max_bytes) return fail(BBP_ERR_OOM, "server_submit: the request alone exceeds the byte budget");
    r->tensors.assign((const unsigned char*)tensors, (const unsigned char*)tensors + raw_bytes);
    for (int k = 0; k < n_terms; ++k) {
        TermCopy t;
        t.nsite = terms[k].nsite;
        if (t.nsite < 1 || t.nsite > 2) return fail(BBP_ERR_INVALID, "server_submit: term must have 1 or 2 sites");
        for (int j = 0; j < t.nsite; ++j) {
            if (!terms[k].op_re[j]) return fail(BBP_ERR_INVALID, "server_submit: operator is NULL");
            t.site[j] = terms[k].site[j];
            const size_t n = op_entries(*desc, t.site[j]);
            if (n == 0) return fail(BBP_ERR_INVALID, "server_submit: site out of range");
            t.re[j].assign(terms[k].op_re[j], terms[k].op_re[j] + n);
            if (terms[k].op_im[j]) {
                t.im[j].assign(terms[k].op_im[j], terms[k].op_im[j] + n);
                t.has_im[j] = true;
            }
        }
        r->terms.push_back(std::move(t));
    }
    std::lock_guard<std::mutex> g(s->mu);
    r->id = s->next_id++;
    r->t_submit = now_s();
    *id = r->id;
    s->queue.push_back(r.get());
    s->reqs[r->id] = std::move(r);
    s->cv_work.notify_one();
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_server_poll(bbp_server* s, long long id, int* state, double* out_re, double* out_im, int* sweeps,
                    double* residual, double* latency_s) try {
    if (!s) return fail(BBP_ERR_INVALID, "server_poll: server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(BBP_ERR_INVALID, "server_poll: unknown request");
    Request* r = it->second.get();
    if (state) *state = r->state;
    if (r->state == 2) {
        for (size_t k = 0; k < r->out_re.size(); ++k) {
            if (out_re) out_re[k] = r->out_re[k];
            if (out_im) out_im[k] = r->out_im[k];
        }
    }
    if (sweeps) *sweeps = r->sweeps;
    if (residual) *residual = r->residual;
    if (latency_s) *latency_s = r->state == 2 || r->state < 0 ? r->t_finish - r->t_submit : 0.0;
    if (r->state < 0) g_err = r->error;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_server_wait(bbp_server* s, long long id, double timeout_s) try {
    if (!s) return fail(BBP_ERR_INVALID, "server_wait: server is NULL");
    if (!(timeout_s >= 0.0)) return fail(BBP_ERR_INVALID, "server_wait: timeout must be >= 0");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(BBP_ERR_INVALID, "server_wait: unknown request");
    Request* r = it->second.get();
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [r] { return r->state == 2 || r->state < 0; });
    if (!ok) return fail(BBP_ERR_TIMEOUT, "server_wait: request still running");
    if (r->state < 0) {
        g_err = r->error;
        return r->state;
    }
    return BBP_OK;
} catch (...) {
    return abi_error();
}

int bbp_server_stats(bbp_server* s, long long* submitted, long long* done, long long* sweeps, size_t* bytes_in_use) try {
    if (!s) return fail(BBP_ERR_INVALID, "server_stats: server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    long long d = 0;
    for (auto& kv : s->reqs) d += kv.second->state == 2 ? 1 : 0;
    if (submitted) *submitted = (long long)s->reqs.size();
    if (done) *done = d;
    if (sweeps) *sweeps = s->sweeps_total.load();
    if (bytes_in_use) *bytes_in_use = s->used;
    return BBP_OK;
} catch (...) {
    return abi_error();
}

void bbp_server_destroy(bbp_server* s) try {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        // queued requests that never started are dropped
        for (Request* r : s->queue) {
            r->state = BBP_ERR_STATE;
            r->error = "server destroyed before the request started";
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();  // runs the admitted solves to the end
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->ro_stop = true;
    }
    s->cv_ro.notify_all();
    if (s->ro_worker.joinable()) s->ro_worker.join();  // reads out what is left
    delete s;
} catch (...) {
    abi_error();
}

}  // extern "C"
