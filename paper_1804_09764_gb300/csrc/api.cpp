// api.cpp -- the extern "C" entry points declared in include/cc.h.
#include <algorithm>
#include <cstring>
#include <vector>

#include "runtime.h"

namespace cc {

static thread_local std::string t_err = "no error";

cc_status fail(cc_status s, const std::string &msg)
{
    t_err = msg;
    return s;
}

}  // namespace cc

using namespace cc;

extern "C" {

const char *cc_version(void) { return "cc-gb300 0.1 (sm_103a)"; }

const char *cc_last_error(void) { return t_err.c_str(); }

const char *cc_status_string(cc_status s)
{
    switch (s) {
    case CC_OK: return "CC_OK";
    case CC_PENDING: return "CC_PENDING";
    case CC_ERR_INVALID_ARG: return "CC_ERR_INVALID_ARG";
    case CC_ERR_BAD_GRAPH: return "CC_ERR_BAD_GRAPH";
    case CC_ERR_NOT_TREE: return "CC_ERR_NOT_TREE";
    case CC_ERR_K_RANGE: return "CC_ERR_K_RANGE";
    case CC_ERR_BUDGET: return "CC_ERR_BUDGET";
    case CC_ERR_WIDTH: return "CC_ERR_WIDTH";
    case CC_ERR_CUDA: return "CC_ERR_CUDA";
    case CC_ERR_TIMEOUT: return "CC_ERR_TIMEOUT";
    case CC_ERR_CANCELLED: return "CC_ERR_CANCELLED";
    case CC_ERR_NOT_FOUND: return "CC_ERR_NOT_FOUND";
    case CC_ERR_CAPACITY: return "CC_ERR_CAPACITY";
    case CC_ERR_NO_MEMORY: return "CC_ERR_NO_MEMORY";
    case CC_ERR_INTERNAL: return "CC_ERR_INTERNAL";
    default: return "CC_UNKNOWN_STATUS";
    }
}

void cc_default_options(cc_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->device = 0;
    opt->width_bits = 0;
    opt->split_threshold = 0;
    opt->batch = 0;
    opt->block_vertices = 0;
    opt->use_cuda_graph = 0;
    opt->fused = 1;
    opt->autotune = 0;
    opt->max_slots = 4;
    opt->timing = 0;
    opt->gather_mode = 1;
}

cc_status cc_create(cc_ctx **out, const cc_options *opt)
{
    if (!out) return fail(CC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    auto c = new (std::nothrow) Ctx();
    if (!c) return fail(CC_ERR_NO_MEMORY, "host allocation failed");
    if (opt)
        c->opt = *opt;
    else
        cc_default_options(&c->opt);
    if (c->opt.max_slots <= 0) c->opt.max_slots = 4;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        delete c;
        return fail(CC_ERR_CUDA, "no CUDA device available");
    }
    if (c->opt.device < 0 || c->opt.device >= ndev) {
        delete c;
        return fail(CC_ERR_INVALID_ARG, "device ordinal out of range");
    }
    c->device = c->opt.device;
    if (cudaSetDevice(c->device) != cudaSuccess) {
        delete c;
        return fail(CC_ERR_CUDA, "cudaSetDevice failed");
    }
    if (c->opt.stream) {
        c->stream = (cudaStream_t)c->opt.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(CC_ERR_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    if (c->opt.l2_persist_mb > 0) {
        // set-aside L2 for persisting accesses (this context only) and the
        // access window the table gathers will use
        int max_persist = 0, max_window = 0;
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, c->device);
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, c->device);
        const uint64_t want = (uint64_t)c->opt.l2_persist_mb << 20;
        const uint64_t setaside = std::min<uint64_t>(want, (uint64_t)std::max(0, max_persist));
        if (setaside > 0 && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, setaside) == cudaSuccess)
            c->l2_window_bytes = std::min<uint64_t>(setaside, (uint64_t)std::max(0, max_window));
        cudaGetLastError();
    }
    uint64_t bytes = c->opt.hbm_budget_bytes;
    if (c->opt.arena) {
        if (!bytes) {
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return fail(CC_ERR_INVALID_ARG, "arena given without hbm_budget_bytes");
        }
        c->arena_base = (char *)c->opt.arena;
    } else {
        if (!bytes) {
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            bytes = (uint64_t)(fr * 0.9);
        }
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return fail(CC_ERR_BUDGET, "could not allocate the HBM arena");
        }
        c->arena_base = (char *)p;
        c->own_arena = true;
    }
    c->arena.init(c->arena_base, bytes);
    c->timer.on = c->opt.timing != 0;
    init_kernel_attributes();
    *out = reinterpret_cast<cc_ctx *>(c);
    return CC_OK;
}

cc_status cc_destroy(cc_ctx *ctx)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    serve_shutdown(c);
    {
        std::lock_guard<std::recursive_mutex> lk(c->mu);
        cudaSetDevice(c->device);
        cudaStreamSynchronize(c->stream);
        evict_plans(c);
        for (auto &kv : c->graphs) graph_free(c, kv.second.get());
        c->graphs.clear();
        for (auto e : c->timer.pool) cudaEventDestroy(e);
        for (auto &q : c->timer.pending) {
            cudaEventDestroy(q.a);
            cudaEventDestroy(q.b);
        }
        if (c->own_arena) cudaFree(c->arena_base);
        if (c->own_stream) cudaStreamDestroy(c->stream);
    }
    delete c;
    return CC_OK;
}

cc_status cc_graph_load_csr(cc_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                            cc_graph_id *out)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return graph_load(c, n, row_ptr, col_idx, flags, out);
}

cc_status cc_graph_load_batch(cc_ctx *ctx, int32_t n_graphs, const int64_t *member_off, int64_t n,
                              const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags, cc_graph_id *out)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    if (n_graphs < 1 || !member_off) return fail(CC_ERR_INVALID_ARG, "n_graphs < 1 or member_off is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return graph_load(c, n, row_ptr, col_idx, flags, out, n_graphs, member_off);
}

cc_status cc_graph_members(cc_ctx *ctx, cc_graph_id g, int32_t *n_graphs)
{
    if (!ctx || !n_graphs) return fail(CC_ERR_INVALID_ARG, "ctx or n_graphs is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    auto it = c->graphs.find(g);
    if (it == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    *n_graphs = it->second->n_members;
    return CC_OK;
}

cc_status cc_graph_free(cc_ctx *ctx, cc_graph_id g)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    auto it = c->graphs.find(g);
    if (it == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    if (it->second->in_use) return fail(CC_ERR_INVALID_ARG, "graph is used by a queued or running request");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    evict_plans(c, g, -1);
    graph_free(c, it->second.get());
    c->graphs.erase(it);
    return CC_OK;
}

static cc_status template_load(cc_ctx *ctx, int32_t k, const int32_t *edges, const uint8_t *labels, int32_t root,
                               cc_template_id *out)
{
    if (!ctx || !out) return fail(CC_ERR_INVALID_ARG, "ctx or out is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    TemplatePlan tp;
    std::string err;
    int rc = build_template_plan(k, edges, root, 1, 16.0, &tp, &err, labels);
    if (rc) return fail(rc, err);
    auto t = std::make_unique<Template>();
    t->k = k;
    t->root_req = root;
    if (k > 1) t->edges.assign(edges, edges + 2 * (k - 1));
    if (labels) t->labels.assign(labels, labels + k);
    t->aut = tp.aut;
    std::vector<std::vector<int>> adj(k);
    for (int i = 0; i + 1 < k; i++) {
        adj[edges[2 * i]].push_back(edges[2 * i + 1]);
        adj[edges[2 * i + 1]].push_back(edges[2 * i]);
    }
    t->canon = tree_canonical_form(k, adj, labels);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    int64_t id = c->next_id++;
    c->templates[id] = std::move(t);
    *out = id;
    return CC_OK;
}

cc_status cc_template_load(cc_ctx *ctx, int32_t k, const int32_t *edges, int32_t root, cc_template_id *out)
{
    return template_load(ctx, k, edges, nullptr, root, out);
}

cc_status cc_template_load_labelled(cc_ctx *ctx, int32_t k, const int32_t *edges, const uint8_t *labels,
                                    int32_t root, cc_template_id *out)
{
    if (!labels) return fail(CC_ERR_INVALID_ARG, "labels is NULL");
    return template_load(ctx, k, edges, labels, root, out);
}

cc_status cc_graph_set_labels(cc_ctx *ctx, cc_graph_id g, const uint8_t *labels)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    auto it = c->graphs.find(g);
    if (it == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    Graph *G = it->second.get();
    if (G->in_use) return fail(CC_ERR_INVALID_ARG, "graph is used by a queued or running request");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    evict_plans(c, g);  // cached plans and captured passes hold the label pointer
    c->arena.free(G->labels);
    G->labels = nullptr;
    G->h_labels.clear();
    if (!labels) return CC_OK;
    G->h_labels.assign(labels, labels + G->n);
    std::vector<uint8_t> lc(std::max<int64_t>(G->n_act, 1), 0);
    for (int64_t v = 0; v < G->n; v++)
        if (G->h_new_id[v] >= 0) lc[G->h_new_id[v]] = labels[v];
    G->labels = (uint8_t *)arena_alloc(c, lc.size());
    if (!G->labels) {
        G->h_labels.clear();
        return fail(CC_ERR_BUDGET, "no room for the vertex labels");
    }
    CC_CUDA(cudaMemcpyAsync(G->labels, lc.data(), lc.size(), cudaMemcpyHostToDevice, c->stream));
    CC_CUDA(cudaStreamSynchronize(c->stream));
    return CC_OK;
}

cc_status cc_template_free(cc_ctx *ctx, cc_template_id t)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    if (!c->templates.count(t)) return fail(CC_ERR_NOT_FOUND, "unknown template");
    evict_plans(c, -1, t);
    c->templates.erase(t);
    return CC_OK;
}

cc_status cc_count(cc_ctx *ctx, cc_graph_id g, cc_template_id t, uint64_t seed, int32_t n_iter, uint64_t *counts,
                   int32_t limbs_capacity, cc_result *res)
{
    cc_count_args a;
    std::memset(&a, 0, sizeof a);
    a.seed = seed;
    a.n_iter = n_iter;
    a.mom_groups = 1;
    a.width_bits = -1;
    return cc_count_ex(ctx, g, t, &a, counts, limbs_capacity, res);
}

cc_status cc_count_ex(cc_ctx *ctx, cc_graph_id g, cc_template_id t, const cc_count_args *args, uint64_t *counts,
                      int32_t limbs_capacity, cc_result *res)
{
    if (!ctx || !args) return fail(CC_ERR_INVALID_ARG, "ctx or args is NULL");
    if (args->n_iter < 0 || limbs_capacity < 1) return fail(CC_ERR_INVALID_ARG, "n_iter < 0 or limbs_capacity < 1");
    if (args->n_sample < 0 || (args->n_sample > 0 && !args->sample_vertices))
        return fail(CC_ERR_INVALID_ARG, "bad sample vertex list");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    CountJob job;
    job.seed = args->seed;
    job.first_iter = args->first_iter;
    job.n_iter = args->n_iter;
    job.mom_groups = args->mom_groups > 0 ? args->mom_groups : 1;
    job.width_bits = args->width_bits;
    if (args->n_sample > 0) job.sample_vertices.assign(args->sample_vertices, args->sample_vertices + args->n_sample);
    if (res) std::memset(res, 0, sizeof *res);
    return count_sync(c, g, t, job, counts, limbs_capacity, args->maps,
                      args->n_sample > 0 ? args->sample_maps : nullptr, res);
}

cc_status cc_count_batch(cc_ctx *ctx, cc_graph_id g, cc_template_id t, const cc_count_args *args, uint64_t *counts,
                         int32_t limbs_capacity, double *estimates, cc_result *res)
{
    if (!ctx || !args) return fail(CC_ERR_INVALID_ARG, "ctx or args is NULL");
    if (args->n_iter < 0 || limbs_capacity < 1) return fail(CC_ERR_INVALID_ARG, "n_iter < 0 or limbs_capacity < 1");
    if (args->n_sample < 0 || (args->n_sample > 0 && !args->sample_vertices))
        return fail(CC_ERR_INVALID_ARG, "bad sample vertex list");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    auto git = c->graphs.find(g);
    if (git == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    CountJob job;
    job.seed = args->seed;
    job.first_iter = args->first_iter;
    job.n_iter = args->n_iter;
    job.mom_groups = args->mom_groups > 0 ? args->mom_groups : 1;
    job.width_bits = args->width_bits;
    if (args->n_sample > 0) job.sample_vertices.assign(args->sample_vertices, args->sample_vertices + args->n_sample);
    std::vector<double> est(git->second->n_members);
    if (res) std::memset(res, 0, sizeof *res);
    cc_status rc = count_sync(c, g, t, job, counts, limbs_capacity, args->maps,
                              args->n_sample > 0 ? args->sample_maps : nullptr, res, est.data());
    if (rc == CC_OK && estimates) std::copy(est.begin(), est.end(), estimates);
    return rc;
}

cc_status cc_count_multi(cc_ctx *ctx, cc_graph_id g, const cc_template_id *tmpls, int32_t n_tmpl,
                         const cc_count_args *args, uint64_t *counts, int32_t limbs_capacity, cc_result *res)
{
    if (!ctx || !args || !tmpls || n_tmpl < 1) return fail(CC_ERR_INVALID_ARG, "ctx, args or templates missing");
    if (args->n_iter < 0 || limbs_capacity < 1) return fail(CC_ERR_INVALID_ARG, "n_iter < 0 or limbs_capacity < 1");
    if (args->n_sample != 0) return fail(CC_ERR_INVALID_ARG, "sampled vertices need a single template");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    CountJob job;
    job.seed = args->seed;
    job.first_iter = args->first_iter;
    job.n_iter = args->n_iter;
    job.mom_groups = args->mom_groups > 0 ? args->mom_groups : 1;
    job.width_bits = args->width_bits;
    if (res) std::memset(res, 0, sizeof *res * n_tmpl);
    return count_multi_sync(c, g, std::vector<int64_t>(tmpls, tmpls + n_tmpl), job, counts, limbs_capacity,
                            args->maps, res);
}

cc_status cc_multi_plan_info_get(cc_ctx *ctx, cc_graph_id g, const cc_template_id *tmpls, int32_t n_tmpl,
                                 int32_t n_iter, cc_multi_info *out)
{
    if (!ctx || !tmpls || n_tmpl < 1 || !out || n_iter < 1) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    std::unique_ptr<PlanInstance> p;
    cc_status rc = make_plan_multi(c, g, std::vector<int64_t>(tmpls, tmpls + n_tmpl), n_iter,
                                   c->opt.width_bits, c->stream, &p);
    if (rc != CC_OK) return rc;
    std::memset(out, 0, sizeof *out);
    out->chains = (int32_t)p->tp.chains.size();
    out->chains_separate = p->sep_chains;
    out->updates_per_colouring = p->updates;
    out->updates_per_colouring_separate = p->sep_updates;
    out->workspace_bytes = p->ws_bytes;
    out->batch = p->B;
    free_plan(c, p.get());
    return CC_OK;
}

cc_status cc_plan_info_get(cc_ctx *ctx, cc_graph_id g, cc_template_id t, cc_plan_info *out)
{
    if (!ctx || !out) return fail(CC_ERR_INVALID_ARG, "ctx or out is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    auto git = c->graphs.find(g);
    auto tit = c->templates.find(t);
    if (git == c->graphs.end() || tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown handle");
    std::memset(out, 0, sizeof *out);
    out->k = tit->second->k;
    out->n_vertices = git->second->n;
    out->n_active = git->second->n_act;
    out->n_directed_edges = git->second->nnz;
    if (tit->second->k == 1 || git->second->n_act == 0) return CC_OK;
    // the plan the last count of (g, t) used, if it is still cached; else a
    // plan for a count of opt.batch (or 16) colourings
    const PlanInstance *cached = nullptr;
    uint64_t last = 0;
    for (auto &kv : c->plan_cache)
        if (std::get<0>(kv.first) == g && std::get<1>(kv.first) == t && std::get<3>(kv.first) == c->opt.width_bits &&
            kv.second.last_use >= last) {
            cached = kv.second.p.get();
            last = kv.second.last_use;
        }
    std::unique_ptr<PlanInstance> own;
    if (!cached) {
        int n_iter = c->opt.batch > 0 ? c->opt.batch : 16;
        CC_TRY(make_plan(c, g, t, n_iter, c->opt.width_bits, c->stream, &own));
    }
    const PlanInstance *p = cached ? cached : own.get();
    out->root = p->tp.root;
    out->n_chains = (int)p->tp.chains.size();
    out->n_tables = out->n_chains - 1;
    out->limbs_root = p->L_root;
    out->batch = p->B;
    out->n_blocks = (int64_t)p->blocks.size();
    out->updates_per_colouring = p->updates;
    out->gather_bytes_per_colouring = p->gather_bytes;
    out->algorithmic_bytes_per_colouring = p->alg_bytes;
    out->pairs_per_colouring = p->pairs;
    out->workspace_bytes = p->ws_bytes;
    out->table4_memory = p->tp.table4_memory;
    out->table4_computation = p->tp.table4_computation;
    out->limb_products_per_colouring = p->limb_products;
    out->split_threshold = p->split;
    out->block_vertices = p->V;
    out->col_chunks = p->col_chunks;
    out->shape_tuned = p->shape_tuned ? 1 : 0;
    out->workspace_no_reuse_bytes = p->ws_no_reuse;
    out->workspace_no_blocks_bytes = p->ws_no_blocks;
    out->workspace_naive_bytes = p->ws_naive;
    if (own) free_plan(c, own.get());
    return CC_OK;
}

cc_status cc_plan_steps_get(cc_ctx *ctx, cc_graph_id g, cc_template_id t, cc_step_info *out, int32_t cap,
                            int32_t *n_steps)
{
    if (!ctx || !n_steps || cap < 0 || (cap > 0 && !out)) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    auto git = c->graphs.find(g);
    auto tit = c->templates.find(t);
    if (git == c->graphs.end() || tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown handle");
    *n_steps = 0;
    if (tit->second->k == 1 || git->second->n_act == 0) return CC_OK;
    const PlanInstance *cached = nullptr;
    uint64_t last = 0;
    for (auto &kv : c->plan_cache)
        if (std::get<0>(kv.first) == g && std::get<1>(kv.first) == t && std::get<3>(kv.first) == c->opt.width_bits &&
            kv.second.last_use >= last) {
            cached = kv.second.p.get();
            last = kv.second.last_use;
        }
    std::unique_ptr<PlanInstance> own;
    if (!cached) {
        int n_iter = c->opt.batch > 0 ? c->opt.batch : 16;
        CC_TRY(make_plan(c, g, t, n_iter, c->opt.width_bits, c->stream, &own));
    }
    const PlanInstance *p = cached ? cached : own.get();
    int32_t n = 0;
    for (size_t ci = 0; ci < p->tp.chains.size(); ci++) {
        const ChainPlan &C = p->tp.chains[ci];
        for (size_t si = 0; si < C.steps.size(); si++, n++) {
            if (n >= cap) continue;
            const Step &st = C.steps[si];
            cc_step_info &r = out[n];
            std::memset(&r, 0, sizeof r);
            r.chain = (int32_t)ci;
            r.step = (int32_t)si;
            r.vertex = C.vertex;
            r.child = st.child;
            r.h = st.h;
            r.a = st.a;
            r.p = st.p;
            r.src_chain = st.src_chain;
            r.is_root = C.is_root ? 1 : 0;
            r.limbs = p->step_L[ci][si];
            r.agg_limbs = p->agg_L[ci][si];
            r.src_limbs = st.src_chain >= 0 ? p->chain_L[st.src_chain] : 0;
            r.chain_limbs = p->chain_L[ci];
            if (ci < p->step_path.size() && si < p->step_path[ci].size()) {
                const auto &sp = p->step_path[ci][si];
                r.path = sp.path;
                r.kernel_limbs[0] = sp.l0;
                r.kernel_limbs[1] = sp.l1;
                r.kernel_limbs[2] = sp.l2;
            }
        }
    }
    *n_steps = n;
    if (own) free_plan(c, own.get());
    return CC_OK;
}

cc_status cc_kernel_instance_stats_get(cc_ctx *ctx, cc_instance_stats *out, int32_t cap, int32_t *n)
{
    if (!ctx || cap < 0 || (cap > 0 && !out)) return fail(CC_ERR_INVALID_ARG, "bad arguments");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    int32_t rows = 0;
    for (int kind = 0; kind < CC_KERNEL_KINDS; kind++)
        for (const auto &kv : c->timer.instances[kind]) {
            if (rows < cap) {
                cc_instance_stats &r = out[rows];
                std::memset(&r, 0, sizeof r);
                std::strncpy(r.name, kv.first.c_str(), sizeof r.name - 1);
                r.kind = kind;
                r.launches = kv.second.launches;
                r.timed_launches = kv.second.timed_launches;
                r.seconds = kv.second.seconds;
                r.bytes = kv.second.bytes;
            }
            rows++;
        }
    if (n) *n = rows;
    return CC_OK;
}

cc_status cc_kernel_stats_get(cc_ctx *ctx, cc_kernel_stats *out)
{
    if (!ctx || !out) return fail(CC_ERR_INVALID_ARG, "ctx or out is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    static const char *names[CC_KERNEL_KINDS] = {"colour", "hist", "gather", "combine", "reduce", "fused", "select", "combine_hist", "heavy"};
    std::memset(out, 0, sizeof *out);
    for (int i = 0; i < CC_KERNEL_KINDS; i++) {
        out->name[i] = names[i];
        out->launches[i] = c->timer.launches[i];
        out->seconds[i] = c->timer.seconds[i];
        out->bytes[i] = c->timer.bytes[i];
    }
    out->total_launches = c->launches.load();
    return CC_OK;
}

cc_status cc_kernel_stats_reset(cc_ctx *ctx)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    for (int i = 0; i < CC_KERNEL_KINDS; i++) {
        c->timer.launches[i] = 0;
        c->timer.seconds[i] = 0;
        c->timer.bytes[i] = 0;
        c->timer.instances[i].clear();
    }
    c->launches = 0;
    return CC_OK;
}

cc_status cc_template_cost(int32_t k, const int32_t *edges, int32_t root, int32_t order, int64_t *memory,
                           int64_t *computation)
{
    if (!memory || !computation) return fail(CC_ERR_INVALID_ARG, "NULL output");
    if (root < 0) return fail(CC_ERR_INVALID_ARG, "root must be given");
    TemplatePlan tp;
    std::string err;
    int rc = build_template_plan(k, edges, root, order == 1 ? 1 : 0, 16.0, &tp, &err);
    if (rc) return fail(rc, err);
    *memory = tp.table4_memory;
    *computation = tp.table4_computation;
    return CC_OK;
}

cc_status cc_template_automorphisms_labelled(int32_t k, const int32_t *edges, const uint8_t *labels, int64_t *aut)
{
    if (!aut || !labels) return fail(CC_ERR_INVALID_ARG, "aut or labels is NULL");
    TemplatePlan tp;
    std::string err;
    int rc = build_template_plan(k, edges, 0, 0, 16.0, &tp, &err, labels);
    if (rc) return fail(rc, err);
    *aut = tp.aut;
    return CC_OK;
}

cc_status cc_limb_product_rate(cc_ctx *ctx, double *per_second)
{
    if (!ctx || !per_second) return fail(CC_ERR_INVALID_ARG, "ctx or per_second is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    uint64_t *scratch = (uint64_t *)arena_alloc(c, 256);
    if (!scratch) return fail(CC_ERR_BUDGET, "no room for one word");
    *per_second = limb_product_rate(c->stream, scratch);
    c->arena.free(scratch);
    c->launches += 2;
    if (*per_second <= 0) return fail(CC_ERR_CUDA, "limb product rate kernel failed");
    return CC_OK;
}

cc_status cc_template_canonical_form(int32_t k, const int32_t *edges, const uint8_t *labels, char *out, int32_t cap)
{
    if (!out) return fail(CC_ERR_INVALID_ARG, "out is NULL");
    TemplatePlan tp;
    std::string err;
    int rc = build_template_plan(k, edges, 0, 0, 16.0, &tp, &err, labels);  // validates the tree
    if (rc) return fail(rc, err);
    std::vector<std::vector<int>> adj(k);
    for (int i = 0; i + 1 < k; i++) {
        adj[edges[2 * i]].push_back(edges[2 * i + 1]);
        adj[edges[2 * i + 1]].push_back(edges[2 * i]);
    }
    const std::string f = tree_canonical_form(k, adj, labels);
    if (cap < (int32_t)f.size() + 1) return fail(CC_ERR_CAPACITY, "needs " + std::to_string(f.size() + 1) + " bytes");
    std::memcpy(out, f.c_str(), f.size() + 1);
    return CC_OK;
}

cc_status cc_template_automorphisms(int32_t k, const int32_t *edges, int64_t *aut)
{
    if (!aut) return fail(CC_ERR_INVALID_ARG, "aut is NULL");
    TemplatePlan tp;
    std::string err;
    int rc = build_template_plan(k, edges, 0, 0, 16.0, &tp, &err);
    if (rc) return fail(rc, err);
    *aut = tp.aut;
    return CC_OK;
}

cc_status cc_table_gather(cc_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X,
                          uint64_t *agg, int64_t values, int32_t limbs, int32_t split_threshold)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return table_gather(c, n, row_ptr, col_idx, X, agg, values, limbs, split_threshold);
}

cc_status cc_submit(cc_ctx *ctx, const cc_request *req, cc_req_id *out)
{
    if (!ctx || !req || !out) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    return serve_submit(reinterpret_cast<Ctx *>(ctx), req, out);
}

cc_status cc_poll(cc_ctx *ctx, cc_req_id id, cc_result *res, uint64_t *counts, int32_t limbs_capacity)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    return serve_poll(reinterpret_cast<Ctx *>(ctx), id, res, counts, limbs_capacity, false, 0);
}

cc_status cc_wait(cc_ctx *ctx, cc_req_id id, int64_t timeout_ns, cc_result *res, uint64_t *counts,
                  int32_t limbs_capacity)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    return serve_poll(reinterpret_cast<Ctx *>(ctx), id, res, counts, limbs_capacity, true, timeout_ns);
}

cc_status cc_cancel(cc_ctx *ctx, cc_req_id id)
{
    if (!ctx) return fail(CC_ERR_INVALID_ARG, "ctx is NULL");
    return serve_cancel(reinterpret_cast<Ctx *>(ctx), id);
}

cc_status cc_serve_stats_get(cc_ctx *ctx, cc_serve_stats *out)
{
    if (!ctx || !out) return fail(CC_ERR_INVALID_ARG, "NULL argument");
    return serve_stats(reinterpret_cast<Ctx *>(ctx), out);
}

}  // extern "C"
