// serve.cpp -- continuous-batching serving loop.
//
// Requests (graph, template, seed, colourings) arrive at any time.  A worker
// thread admits the head of the queue when a slot is free and the request's
// plan workspace fits the free arena; every admitted request owns a CUDA
// stream and advances one colouring pass at a time, so passes of different
// requests overlap on the device and a new request starts as soon as memory
// and a slot free up.  Results are bit-identical to cc_count (same plan, same
// kernels, exact integer arithmetic).
#include <algorithm>
#include <chrono>
#include <cstring>

#include "runtime.h"

namespace cc {

using Clock = std::chrono::steady_clock;

struct Request {
    cc_req_id id = 0;
    cc_request req{};
    CountJob job;
    Clock::time_point t_submit, t_done;
    enum State { QUEUED, RUNNING, DONE } state = QUEUED;
    cc_status status = CC_OK;
    std::string error;
    bool cancel = false;
    std::unique_ptr<PlanInstance> plan;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int next_pass = 0, npass = 0;
    bool inflight = false;
    ColourParams *hp = nullptr;
    uint64_t *ht = nullptr;
    cc_result res{};
    std::vector<uint64_t> counts;
};

struct Server {
    Ctx *c = nullptr;
    std::thread th;
    std::mutex m;
    std::condition_variable cv, done_cv;
    bool stop = false;
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::map<cc_req_id, std::unique_ptr<Request>> all;
    std::vector<cudaStream_t> streams;
    std::vector<double> latencies;
    cc_serve_stats st{};
    Clock::time_point busy_since;
    bool busy = false;
    int64_t next_id = 1;
};

Ctx::Ctx() = default;
Ctx::~Ctx() = default;

namespace {

void release(Ctx *c, Server *s, Request *r)
{
    if (r->stream) cudaStreamSynchronize(r->stream);
    c->arena.free(r->ws);
    r->ws = nullptr;
    if (r->plan) free_plan(c, r->plan.get());
    r->plan.reset();
    if (r->hp) cudaFreeHost(r->hp);
    if (r->ht) cudaFreeHost(r->ht);
    r->hp = nullptr;
    r->ht = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    if (r->stream) s->streams.push_back(r->stream);
    r->stream = nullptr;
    auto git = c->graphs.find(r->req.graph);
    if (git != c->graphs.end()) git->second->in_use--;
}

void complete(Ctx *c, Server *s, Request *r, cc_status status, const std::string &err)
{
    release(c, s, r);
    r->status = status;
    r->error = err;
    r->state = Request::DONE;
    r->t_done = Clock::now();
    double lat = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    r->res.wall_seconds = lat;
    if (status == CC_OK) {
        s->st.completed++;
        s->latencies.push_back(lat);
    } else if (status == CC_ERR_CANCELLED) {
        s->st.cancelled++;
    } else {
        s->st.failed++;
    }
    s->done_cv.notify_all();
}

// try to admit r; returns false if it must wait for memory
bool admit(Ctx *c, Server *s, Request *r)
{
    cudaStream_t stream;
    if (!s->streams.empty()) {
        stream = s->streams.back();
        s->streams.pop_back();
    } else if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    r->stream = stream;
    auto git = c->graphs.find(r->req.graph);
    auto tit = c->templates.find(r->req.tmpl);
    if (git == c->graphs.end() || tit == c->templates.end()) {
        git = c->graphs.end();
        r->req.graph = -1;
        complete(c, s, r, CC_ERR_NOT_FOUND, "unknown graph or template");
        return true;
    }
    git->second->in_use++;
    if (tit->second->k == 1 || git->second->n_act == 0 || r->job.n_iter == 0) {
        // no DP: same host-side answer as cc_count
        std::vector<uint64_t> cnt(std::max(1, r->job.n_iter) * 1);
        cc_count_args a{};
        (void)a;
        r->counts.assign(std::max(1, r->job.n_iter), 0);
        uint64_t v = tit->second->k == 1 ? (uint64_t)git->second->n : 0;
        for (auto &x : r->counts) x = v;
        std::memset(&r->res, 0, sizeof r->res);
        r->res.k = tit->second->k;
        r->res.limbs = 1;
        r->res.exact = 1;
        r->res.n_iter = r->job.n_iter;
        r->res.aut = tit->second->aut;
        complete(c, s, r, CC_OK, "");
        return true;
    }
    std::unique_ptr<PlanInstance> p;
    cc_status rc = make_plan(c, r->req.graph, r->req.tmpl, r->job.n_iter, c->opt.width_bits, stream, &p);
    if (rc == CC_ERR_BUDGET && !c->plan_cache.empty()) {
        evict_plans(c);  // plans cached by cc_count give way to served requests
        rc = make_plan(c, r->req.graph, r->req.tmpl, r->job.n_iter, c->opt.width_bits, stream, &p);
    }
    if (rc == CC_ERR_BUDGET && !s->active.empty()) {
        git->second->in_use--;
        s->streams.push_back(stream);
        r->stream = nullptr;
        return false;
    }
    if (rc != CC_OK) {
        complete(c, s, r, rc, cc_last_error());
        return true;
    }
    r->ws = (char *)arena_alloc(c, p->ws_bytes);
    if (!r->ws) {
        free_plan(c, p.get());
        if (!s->active.empty()) {
            git->second->in_use--;
            s->streams.push_back(stream);
            r->stream = nullptr;
            return false;
        }
        r->plan = std::move(p);
        complete(c, s, r, CC_ERR_BUDGET, "workspace does not fit the HBM budget");
        return true;
    }
    r->plan = std::move(p);
    r->plan->tuned = true;  // served passes use the tuned variants if a count tuned them, else the defaults
    r->npass = (r->job.n_iter + r->plan->B - 1) / r->plan->B;
    if (cudaMallocHost(&r->hp, sizeof(ColourParams) * r->npass) != cudaSuccess ||
        cudaMallocHost(&r->ht, (size_t)8 * r->npass * r->plan->B * r->plan->L_root * r->plan->n_slots) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        complete(c, s, r, CC_ERR_CUDA, "pinned buffer or event creation failed");
        return true;
    }
    if (cudaMemsetAsync(r->ws + r->plan->off_err, 0, 256, stream) != cudaSuccess) {
        cudaGetLastError();
        complete(c, s, r, CC_ERR_CUDA, "workspace clear failed");
        return true;
    }
    r->state = Request::RUNNING;
    s->active.push_back(r);
    return true;
}

void worker(Server *s)
{
    Ctx *c = s->c;
    cudaSetDevice(c->device);
    while (true) {
        bool progress = false;
        {
            std::lock_guard<std::recursive_mutex> lc(c->mu);
            std::unique_lock<std::mutex> lk(s->m);
            if (s->stop) break;
            // admission (FIFO; a request that does not fit waits for memory)
            while (!s->queue.empty() && (int)s->active.size() < c->opt.max_slots) {
                Request *r = s->queue.front();
                if (r->cancel) {
                    s->queue.pop_front();
                    r->state = Request::DONE;
                    r->status = CC_ERR_CANCELLED;
                    r->t_done = Clock::now();
                    s->st.cancelled++;
                    s->done_cv.notify_all();
                    progress = true;
                    continue;
                }
                if (!admit(c, s, r)) {
                    s->st.admissions_deferred++;
                    break;
                }
                s->queue.pop_front();
                progress = true;
            }
            // advance every running request by one pass when its previous pass is done
            for (size_t i = 0; i < s->active.size();) {
                Request *r = s->active[i];
                if (r->inflight) {
                    cudaError_t q = cudaEventQuery(r->ev);
                    if (q == cudaErrorNotReady) {
                        i++;
                        continue;
                    }
                    r->inflight = false;
                    if (q != cudaSuccess) {
                        s->active.erase(s->active.begin() + i);
                        complete(c, s, r, CC_ERR_CUDA, cudaGetErrorString(q));
                        progress = true;
                        continue;
                    }
                }
                if (r->cancel) {
                    s->active.erase(s->active.begin() + i);
                    complete(c, s, r, CC_ERR_CANCELLED, "cancelled");
                    progress = true;
                    continue;
                }
                if (r->next_pass < r->npass) {
                    cc_status rc = run_passes(c, r->plan.get(), r->ws, r->job, r->next_pass, r->next_pass + 1,
                                              r->stream, r->hp, r->ht, nullptr, nullptr, 0, nullptr);
                    if (rc == CC_OK && cudaEventRecord(r->ev, r->stream) != cudaSuccess) rc = CC_ERR_CUDA;
                    if (rc != CC_OK) {
                        s->active.erase(s->active.begin() + i);
                        complete(c, s, r, rc, cc_last_error());
                        progress = true;
                        continue;
                    }
                    r->next_pass++;
                    r->inflight = true;
                    progress = true;
                    i++;
                    continue;
                }
                // all passes finished
                int kerr = 0;
                if (cudaMemcpy(&kerr, r->ws + r->plan->off_err, sizeof kerr, cudaMemcpyDeviceToHost) == cudaSuccess &&
                    kerr) {
                    s->active.erase(s->active.begin() + i);
                    complete(c, s, r, CC_ERR_TIMEOUT, "a gather kernel wait ran out of time");
                    progress = true;
                    continue;
                }
                Graph *g = c->graphs.at(r->req.graph).get();
                int L = r->plan->L_root;
                r->counts.assign((size_t)r->job.n_iter * L, 0);
                double dev = 0;
                r->res.device_seconds = dev;
                cc_status rc = finish_counts(c, r->plan.get(), g, r->job, r->ht, nullptr, r->counts.data(), L,
                                             nullptr, nullptr, &r->res);
                s->active.erase(s->active.begin() + i);
                complete(c, s, r, rc, rc == CC_OK ? "" : cc_last_error());
                progress = true;
            }
            const bool now_busy = !s->active.empty();
            if (now_busy && !s->busy) s->busy_since = Clock::now();
            if (!now_busy && s->busy)
                s->st.busy_seconds += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
            s->busy = now_busy;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->m);
            if (s->stop) break;
            s->cv.wait_for(lk, std::chrono::microseconds(100));
        }
    }
}

Server *get_server(Ctx *c)
{
    std::lock_guard<std::recursive_mutex> lc(c->mu);
    if (!c->server) {
        c->server = std::make_unique<Server>();
        c->server->c = c;
        c->server->th = std::thread(worker, c->server.get());
    }
    return c->server.get();
}

}  // namespace

cc_status serve_submit(Ctx *c, const cc_request *q, cc_req_id *out)
{
    if (q->n_iter < 0) return fail(CC_ERR_INVALID_ARG, "n_iter < 0");
    {
        std::lock_guard<std::recursive_mutex> lc(c->mu);
        if (!c->graphs.count(q->graph)) return fail(CC_ERR_NOT_FOUND, "unknown graph");
        if (!c->templates.count(q->tmpl)) return fail(CC_ERR_NOT_FOUND, "unknown template");
    }
    Server *s = get_server(c);
    auto r = std::make_unique<Request>();
    r->req = *q;
    r->job.seed = q->seed;
    r->job.first_iter = q->first_iter;
    r->job.n_iter = q->n_iter;
    r->job.mom_groups = 1;
    r->job.width_bits = -1;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->m);
    r->id = s->next_id++;
    *out = r->id;
    s->queue.push_back(r.get());
    s->all[r->id] = std::move(r);
    s->st.submitted++;
    s->cv.notify_all();
    return CC_OK;
}

cc_status serve_poll(Ctx *c, cc_req_id id, cc_result *res, uint64_t *counts, int32_t cap, bool wait, int64_t timeout_ns)
{
    Server *s = get_server(c);
    std::unique_lock<std::mutex> lk(s->m);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(CC_ERR_NOT_FOUND, "unknown request");
    Request *r = it->second.get();
    if (r->state != Request::DONE) {
        if (!wait) return CC_PENDING;
        auto until = Clock::now() + std::chrono::nanoseconds(timeout_ns < 0 ? int64_t(1) << 62 : timeout_ns);
        while (r->state != Request::DONE) {
            if (s->done_cv.wait_until(lk, until) == std::cv_status::timeout && r->state != Request::DONE)
                return fail(CC_ERR_TIMEOUT, "request not finished within the timeout");
        }
    }
    if (r->status != CC_OK) {
        cc_status st = r->status;
        std::string e = r->error;
        s->all.erase(it);
        return fail(st, e.empty() ? "request failed" : e);
    }
    const int L = std::max(1, r->res.limbs);
    if (res) *res = r->res;
    if (counts) {
        if (cap < L) return fail(CC_ERR_CAPACITY, "limbs_capacity too small");
        for (int j = 0; j < r->job.n_iter; j++)
            for (int l = 0; l < cap; l++)
                counts[(size_t)j * cap + l] = l < L ? r->counts[(size_t)j * L + l] : 0;
    }
    s->all.erase(it);
    return CC_OK;
}

cc_status serve_cancel(Ctx *c, cc_req_id id)
{
    Server *s = get_server(c);
    std::lock_guard<std::mutex> lk(s->m);
    auto it = s->all.find(id);
    if (it == s->all.end()) return fail(CC_ERR_NOT_FOUND, "unknown request");
    it->second->cancel = true;
    s->cv.notify_all();
    return CC_OK;
}

cc_status serve_stats(Ctx *c, cc_serve_stats *out)
{
    Server *s = get_server(c);
    std::lock_guard<std::mutex> lk(s->m);
    *out = s->st;
    out->in_flight = (int64_t)s->active.size();
    out->queued = (int64_t)s->queue.size();
    if (s->busy) out->busy_seconds += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
        out->p50_latency_s = q(0.50);
        out->p99_latency_s = q(0.99);
        double sum = 0;
        for (double x : l) sum += x;
        out->mean_latency_s = sum / l.size();
    }
    return CC_OK;
}

void serve_shutdown(Ctx *c)
{
    if (!c->server) return;
    Server *s = c->server.get();
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    std::lock_guard<std::recursive_mutex> lc(c->mu);
    for (Request *r : s->active) release(c, s, r);
    s->active.clear();
    for (auto st : s->streams) cudaStreamDestroy(st);
    s->streams.clear();
    c->server.reset();
}

}  // namespace cc
