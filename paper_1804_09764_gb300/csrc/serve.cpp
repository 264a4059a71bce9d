// serve.cpp -- continuous-batching serving loop.
//
// Requests (graph, template, seed, colourings) arrive at any time and queue.
// A worker thread groups the admitted requests by graph and by template up to
// isomorphism: isomorphic templates have the same copy counts in every
// colouring, so one plan serves every request of a group.  A group owns a
// CUDA stream and a workspace and runs one colouring pass at a time.  A pass
// takes the next pending colourings of all the group's requests, in arrival
// order, up to the batch cap: colourings of different requests sit side by
// side in the pass's colouring parameters (each with its own seed and index),
// so they share every launch of the pass.  Between passes requests join (as
// soon as they are admitted) and leave (when their last colouring is back):
// continuous batching at the granularity of colourings.  The workspace is
// re-planned when the pending colourings call for another batch size.  Groups
// of different graphs or template classes run concurrently on their own
// streams, up to max_slots groups; a new group is admitted when its workspace
// fits the free arena.  A colouring's total depends only on the graph, the
// template class, the seed and the colouring index, so every result is
// bit-identical to cc_count's.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "runtime.h"

namespace cc {

using Clock = std::chrono::steady_clock;

struct Group;

struct Request {
    cc_req_id id = 0;
    cc_request req{};
    CountJob job;
    Clock::time_point t_submit, t_done;
    enum State { QUEUED, RUNNING, DONE } state = QUEUED;
    cc_status status = CC_OK;
    std::string error;
    bool cancel = false;
    bool holds_graph = false;  // counted in the graph's in_use
    Group *group = nullptr;
    int next_j = 0, done_j = 0;  // colourings dispatched / with totals back
    std::vector<uint64_t> maps;  // root totals per colouring (L_root limbs), padded to whole passes
    cc_result res{};
    std::vector<uint64_t> counts;
};

struct Group {
    int64_t graph = 0;
    int64_t tmpl = 0;    // the template its plans use (that of the request that opened it)
    std::string canon;
    int L_root = 0;
    std::unique_ptr<PlanInstance> plan;  // planned for the batch size of the pass
    int planned_for = 0;                 // the batch asked for when planning (the plan's B may be smaller)
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    ColourParams *hp = nullptr;  // pinned: parameters of one pass
    uint64_t *ht = nullptr;      // pinned: totals of one pass
    int32_t *herr = nullptr;     // pinned: the workspace's kernel error word after the pass
    std::vector<Request *> members;                 // arrival order
    std::vector<std::pair<cc_req_id, int>> slots;   // (request, colouring j) of each colouring of the pass in flight
    bool inflight = false;
};

struct Server {
    Ctx *c = nullptr;
    std::thread th;
    std::mutex m;
    std::condition_variable cv, done_cv;
    bool stop = false;
    std::deque<Request *> queue;
    std::vector<std::unique_ptr<Group>> groups;
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

constexpr int kHostTotalsWords = 64 * 4;  // a pass: at most 64 colourings of at most 4 limbs

int batch_cap(const Ctx *c) { return std::max(1, std::min(c->opt.batch > 0 ? c->opt.batch : 16, 64)); }

void complete(Ctx *c, Server *s, Request *r, cc_status status, const std::string &err)
{
    if (r->holds_graph) {
        auto git = c->graphs.find(r->req.graph);
        if (git != c->graphs.end()) git->second->in_use--;
        r->holds_graph = false;
    }
    r->group = nullptr;
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

void free_group_plan(Ctx *c, Group *g)
{
    if (g->stream) cudaStreamSynchronize(g->stream);
    c->arena.free(g->ws);
    g->ws = nullptr;
    if (g->plan) free_plan(c, g->plan.get());
    g->plan.reset();
}

void release_group(Ctx *c, Server *s, Group *g)
{
    free_group_plan(c, g);
    if (g->hp) cudaFreeHost(g->hp);
    if (g->ht) cudaFreeHost(g->ht);
    if (g->herr) cudaFreeHost(g->herr);
    g->hp = nullptr;
    g->ht = nullptr;
    g->herr = nullptr;
    if (g->ev) cudaEventDestroy(g->ev);
    g->ev = nullptr;
    if (g->stream) s->streams.push_back(g->stream);
    g->stream = nullptr;
}

// (Re)plan group g for a pass of `want` colourings (fewer if the budget says
// so).  CC_ERR_BUDGET when not even one colouring fits.
cc_status plan_group(Ctx *c, Group *g, int want)
{
    free_group_plan(c, g);
    const int64_t tid = g->tmpl;
    if (!c->templates.count(tid)) return fail(CC_ERR_NOT_FOUND, "template freed while its requests ran");
    std::unique_ptr<PlanInstance> p;
    cc_status rc = make_plan(c, g->graph, tid, want, c->opt.width_bits, g->stream, &p);
    if (rc == CC_ERR_BUDGET && !c->plan_cache.empty()) {
        evict_plans(c);  // plans cached by cc_count give way to served requests
        rc = make_plan(c, g->graph, tid, want, c->opt.width_bits, g->stream, &p);
    }
    if (rc != CC_OK) return rc;
    char *ws = (char *)arena_alloc(c, p->ws_bytes);
    if (!ws) {
        free_plan(c, p.get());
        return fail(CC_ERR_BUDGET, "workspace does not fit the HBM budget");
    }
    p->tuned = true;  // served passes use the tuned variants if a count tuned them, else the defaults
    CC_CUDA(cudaMemsetAsync(ws + p->off_err, 0, 256, g->stream));
    g->plan = std::move(p);
    g->ws = ws;
    g->L_root = g->plan->L_root;
    return CC_OK;
}

// answer with no DP (k = 1, no edges, no colourings): as cc_count
bool trivial(Request *r, const Template *t, const Graph *g)
{
    if (!(t->k == 1 || g->n_act == 0 || r->job.n_iter == 0)) return false;
    const int n = std::max(1, r->job.n_iter);
    uint64_t v = 0;
    if (t->k == 1) {
        v = (uint64_t)g->n;
        if (!t->labels.empty())
            v = g->h_labels.empty() ? 0 : (uint64_t)std::count(g->h_labels.begin(), g->h_labels.end(), t->labels[0]);
    }
    r->counts.assign(n, v);
    std::memset(&r->res, 0, sizeof r->res);
    r->res.k = t->k;
    r->res.limbs = 1;
    r->res.exact = 1;
    r->res.n_iter = r->job.n_iter;
    r->res.aut = t->aut;
    r->res.estimate = r->res.median_of_means = (double)v;  // k = 1: k^k / k! = 1
    return true;
}

// open a group for request r (its graph and template class); CC_ERR_BUDGET
// when its workspace does not fit now
cc_status open_group(Ctx *c, Server *s, Request *r, const Template *t, std::unique_ptr<Group> *out)
{
    auto ng = std::make_unique<Group>();
    ng->graph = r->req.graph;
    ng->tmpl = r->req.tmpl;
    ng->canon = t->canon;
    if (!s->streams.empty()) {
        ng->stream = s->streams.back();
        s->streams.pop_back();
    } else if (cudaStreamCreateWithFlags(&ng->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ng->stream = nullptr;
        return fail(CC_ERR_CUDA, "stream creation failed");
    }
    // as many colourings per pass as the request has (up to the cap), halved
    // while the workspace does not fit
    const int want = std::min(batch_cap(c), r->job.n_iter);
    cc_status rc = CC_ERR_BUDGET;
    for (int w = want; w >= 1 && rc == CC_ERR_BUDGET; w = w > 1 ? w / 2 : 0) rc = plan_group(c, ng.get(), w);
    ng->planned_for = want;
    if (rc == CC_OK && (cudaMallocHost(&ng->hp, sizeof(ColourParams)) != cudaSuccess ||
                        cudaMallocHost(&ng->ht, (size_t)8 * kHostTotalsWords) != cudaSuccess ||
                        cudaMallocHost(&ng->herr, sizeof(int32_t)) != cudaSuccess ||
                        cudaEventCreateWithFlags(&ng->ev, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        rc = fail(CC_ERR_CUDA, "pinned buffer or event creation failed");
    }
    if (rc != CC_OK) {
        release_group(c, s, ng.get());
        return rc;
    }
    *out = std::move(ng);
    return CC_OK;
}

// Admit queued requests: join the group of their graph and template class, or
// open a group (a slot and workspace permitting).  A request that must wait
// for a slot or memory stops new groups from opening, but later requests may
// still join running groups.
bool admit(Ctx *c, Server *s)
{
    bool progress = false, blocked = false;
    for (size_t qi = 0; qi < s->queue.size();) {
        Request *r = s->queue[qi];
        auto take = [&]() {
            s->queue.erase(s->queue.begin() + qi);
            progress = true;
        };
        if (r->cancel) {
            take();
            r->state = Request::DONE;
            r->status = CC_ERR_CANCELLED;
            r->t_done = Clock::now();
            s->st.cancelled++;
            s->done_cv.notify_all();
            continue;
        }
        auto git = c->graphs.find(r->req.graph);
        auto tit = c->templates.find(r->req.tmpl);
        if (git == c->graphs.end() || tit == c->templates.end()) {
            take();
            complete(c, s, r, CC_ERR_NOT_FOUND, "unknown graph or template");
            continue;
        }
        Graph *g = git->second.get();
        const Template *t = tit->second.get();
        if (trivial(r, t, g)) {
            take();
            complete(c, s, r, CC_OK, "");
            continue;
        }
        Group *gr = nullptr;
        for (auto &x : s->groups)
            if (x->graph == r->req.graph && x->canon == t->canon) gr = x.get();
        if (!gr) {
            if (blocked || (int)s->groups.size() >= std::max(1, c->opt.max_slots)) {
                blocked = true;
                s->st.admissions_deferred++;
                qi++;
                continue;
            }
            std::unique_ptr<Group> ng;
            cc_status rc = open_group(c, s, r, t, &ng);
            if (rc == CC_ERR_BUDGET && !s->groups.empty()) {
                blocked = true;  // running groups will free memory
                s->st.admissions_deferred++;
                qi++;
                continue;
            }
            if (rc != CC_OK) {
                take();
                complete(c, s, r, rc, cc_last_error());
                continue;
            }
            gr = ng.get();
            s->groups.push_back(std::move(ng));
        }
        take();
        r->group = gr;
        r->state = Request::RUNNING;
        r->holds_graph = true;
        g->in_use++;
        r->maps.assign((size_t)(r->job.n_iter + 64) * 4, 0);
        gr->members.push_back(r);
    }
    return progress;
}

// Fold the finished pass of group gr into its requests; requests with all
// their colourings back are finished.
void collect(Ctx *c, Server *s, Group *gr)
{
    const cudaError_t q = cudaEventQuery(gr->ev);
    gr->inflight = false;
    const int L = gr->L_root;
    std::string err;
    cc_status bad = CC_OK;
    if (q != cudaSuccess) {
        bad = CC_ERR_CUDA;
        err = cudaGetErrorString(q);
    } else if (*gr->herr) {
        bad = CC_ERR_TIMEOUT;
        err = "a gather kernel wait ran out of time";
        cudaMemsetAsync(gr->ws + gr->plan->off_err, 0, 256, gr->stream);
    }
    std::vector<cc_req_id> failed;
    for (size_t b = 0; b < gr->slots.size(); b++) {
        const cc_req_id id = gr->slots[b].first;
        auto it = s->all.find(id);
        if (it == s->all.end()) continue;  // cancelled and forgotten
        Request *r = it->second.get();
        if (r->state != Request::RUNNING || r->group != gr) continue;
        if (bad == CC_OK) {
            std::memcpy(&r->maps[(size_t)gr->slots[b].second * L], gr->ht + b * L, 8 * (size_t)L);
            r->done_j++;
        } else if (std::find(failed.begin(), failed.end(), id) == failed.end()) {
            failed.push_back(id);
        }
    }
    gr->slots.clear();
    s->st.passes++;
    for (size_t i = 0; i < gr->members.size();) {
        Request *r = gr->members[i];
        const bool fl = std::find(failed.begin(), failed.end(), r->id) != failed.end();
        if (!fl && r->done_j < r->job.n_iter) {
            i++;
            continue;
        }
        gr->members.erase(gr->members.begin() + i);
        if (fl) {
            complete(c, s, r, bad, err);
            continue;
        }
        // colouring j's total sits at word j * L: the layout finish_counts
        // reads for one root slot and one member (pass ps, colouring b of the
        // pass -> ps * B + b = j)
        Graph *g = c->graphs.at(r->req.graph).get();
        r->counts.assign((size_t)r->job.n_iter * L, 0);
        cc_status rc = finish_counts(c, gr->plan.get(), g, r->job, r->maps.data(), nullptr, r->counts.data(), L,
                                     nullptr, nullptr, &r->res);
        complete(c, s, r, rc, rc == CC_OK ? "" : cc_last_error());
    }
}

void fail_members(Ctx *c, Server *s, Group *gr, cc_status rc)
{
    const std::string e = cc_last_error();
    for (Request *r : gr->members) complete(c, s, r, rc, e);
    gr->members.clear();
    gr->slots.clear();
}

// Start the next pass of group gr: the pending colourings of its requests in
// arrival order, as many as the (re)planned batch takes.  When the pending
// colourings call for another batch size the group is re-planned, halving the
// batch while the workspace does not fit; if not even one colouring fits while
// other groups hold workspace, the group waits for them to give it back.  Returns whether a pass
// was started (or the group's requests finished with an error).
bool launch_next(Ctx *c, Server *s, Group *gr)
{
    int pending = 0;
    for (Request *r : gr->members) pending += r->job.n_iter - r->next_j;
    if (pending <= 0) return false;
    const int want = std::min(batch_cap(c), pending);
    if (!gr->plan || (gr->plan->B != want && gr->planned_for != want)) {
        cc_status rc = CC_ERR_BUDGET;
        for (int w = want; w >= 1 && rc == CC_ERR_BUDGET; w = w > 1 ? w / 2 : 0) rc = plan_group(c, gr, w);
        gr->planned_for = want;
        bool others_hold = false;  // memory that other groups will give back
        for (auto &x : s->groups) others_hold |= x.get() != gr && x->plan != nullptr;
        if (rc == CC_ERR_BUDGET && others_hold) {
            s->st.admissions_deferred++;
            return false;
        }
        if (rc != CC_OK) {
            fail_members(c, s, gr, rc);
            return true;
        }
    }
    PlanInstance *p = gr->plan.get();
    const int B = p->B;  // <= pending: every colouring of the pass belongs to a request
    gr->slots.clear();
    int requests = 0;
    for (Request *r : gr->members) {
        if (r->next_j < r->job.n_iter && (int)gr->slots.size() < B) requests++;
        const uint64_t fs = splitmix64_host(r->job.seed);
        while (r->next_j < r->job.n_iter && (int)gr->slots.size() < B) {
            gr->hp->hj[gr->slots.size()] = splitmix64_host(fs + (uint64_t)(r->job.first_iter + r->next_j));
            gr->slots.push_back({r->id, r->next_j});
            r->next_j++;
        }
    }
    cc_status rc = run_pass_with(c, p, gr->ws, gr->hp, gr->stream, gr->ht);
    if (rc == CC_OK &&
        cudaMemcpyAsync(gr->herr, gr->ws + p->off_err, sizeof(int32_t), cudaMemcpyDeviceToHost, gr->stream) !=
            cudaSuccess)
        rc = fail(CC_ERR_CUDA, "error word read-back failed");
    if (rc == CC_OK && cudaEventRecord(gr->ev, gr->stream) != cudaSuccess) rc = fail(CC_ERR_CUDA, "event record failed");
    if (rc != CC_OK) {
        fail_members(c, s, gr, rc);
        return true;
    }
    gr->inflight = true;
    s->st.colourings_run += B;
    if (requests >= 2) s->st.shared_passes++;
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
            progress |= admit(c, s);
            for (size_t gi = 0; gi < s->groups.size();) {
                Group *gr = s->groups[gi].get();
                if (gr->inflight) {
                    if (cudaEventQuery(gr->ev) == cudaErrorNotReady) {
                        gi++;
                        continue;
                    }
                    collect(c, s, gr);
                    progress = true;
                }
                // cancelled requests leave between passes
                for (size_t i = 0; i < gr->members.size();) {
                    Request *r = gr->members[i];
                    if (r->cancel) {
                        gr->members.erase(gr->members.begin() + i);
                        complete(c, s, r, CC_ERR_CANCELLED, "cancelled");
                        progress = true;
                    } else {
                        i++;
                    }
                }
                if (!gr->members.empty() && launch_next(c, s, gr)) progress = true;
                if (gr->members.empty() && !gr->inflight) {
                    release_group(c, s, gr);
                    s->groups.erase(s->groups.begin() + gi);
                    progress = true;
                    continue;
                }
                gi++;
            }
            const bool now_busy = !s->groups.empty();
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
    int64_t in_flight = 0;
    for (auto &g : s->groups) in_flight += (int64_t)g->members.size();
    out->in_flight = in_flight;
    out->queued = (int64_t)s->queue.size();
    out->groups = (int64_t)s->groups.size();
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
    for (auto &g : s->groups) {
        for (Request *r : g->members)
            if (r->holds_graph) {
                auto git = c->graphs.find(r->req.graph);
                if (git != c->graphs.end()) git->second->in_use--;
                r->holds_graph = false;
            }
        release_group(c, s, g.get());
    }
    s->groups.clear();
    for (auto st : s->streams) cudaStreamDestroy(st);
    s->streams.clear();
    c->server.reset();
}

}  // namespace cc
