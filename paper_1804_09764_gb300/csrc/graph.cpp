// graph.cpp -- loading a CSR graph onto the device, neighbour-list task
// splitting (Algorithm 4), and rooted homomorphism bounds used to size the
// integers of each count table.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "runtime.h"

namespace cc {

namespace {

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cc_status validate_host(int64_t n, const int64_t *rp, const int32_t *ci)
{
    std::vector<int32_t> sorted(ci, ci + rp[n]);
    for (int64_t v = 0; v < n; v++) {
        auto b = sorted.begin() + rp[v], e = sorted.begin() + rp[v + 1];
        for (auto it = b; it != e; ++it) {
            if (*it < 0 || *it >= n) return fail(CC_ERR_BAD_GRAPH, "neighbour id out of range at vertex " + std::to_string(v));
            if (*it == v) return fail(CC_ERR_BAD_GRAPH, "self-loop at vertex " + std::to_string(v));
        }
        std::sort(b, e);
        if (std::adjacent_find(b, e) != e) return fail(CC_ERR_BAD_GRAPH, "duplicate edge at vertex " + std::to_string(v));
    }
    for (int64_t v = 0; v < n; v++)
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            int64_t u = sorted[e];
            if (!std::binary_search(sorted.begin() + rp[u], sorted.begin() + rp[u + 1], (int32_t)v))
                return fail(CC_ERR_BAD_GRAPH, "edge " + std::to_string(v) + "-" + std::to_string(u) +
                                                  " has no reverse direction");
        }
    return CC_OK;
}

}  // namespace

cc_status graph_load(Ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                     cc_graph_id *out, int32_t n_members, const int64_t *member_off)
{
    if (!out) return fail(CC_ERR_INVALID_ARG, "out is NULL");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(CC_ERR_INVALID_ARG, "n out of range");
    if (!row_ptr) return fail(CC_ERR_INVALID_ARG, "row_ptr is NULL");
    if (n_members < 1 || (n_members > 1 && !member_off)) return fail(CC_ERR_INVALID_ARG, "bad member graph count");
    std::vector<int64_t> moff = {0, n};
    if (member_off) {
        moff.assign(member_off, member_off + n_members + 1);
        if (moff[0] != 0 || moff[n_members] != n) return fail(CC_ERR_INVALID_ARG, "member offsets must run from 0 to n");
        for (int32_t i = 0; i < n_members; i++)
            if (moff[i + 1] < moff[i]) return fail(CC_ERR_INVALID_ARG, "member offsets decrease at " + std::to_string(i));
    }
    cudaStream_t st = c->stream;
    auto g = std::make_unique<Graph>();
    g->n = n;
    std::vector<int64_t> rp(n + 1);
    const bool rp_dev = is_device_ptr(row_ptr);
    if (rp_dev) {
        CC_CUDA(cudaMemcpy(rp.data(), row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(rp.data(), row_ptr, sizeof(int64_t) * (n + 1));
    }
    if (rp[0] != 0) return fail(CC_ERR_BAD_GRAPH, "row_ptr[0] must be 0");
    for (int64_t v = 0; v < n; v++)
        if (rp[v + 1] < rp[v]) return fail(CC_ERR_BAD_GRAPH, "row_ptr decreases at " + std::to_string(v));
    const int64_t nnz = rp[n];
    if (nnz > 0 && !col_idx) return fail(CC_ERR_INVALID_ARG, "col_idx is NULL");
    if (nnz >= (int64_t(1) << 40)) return fail(CC_ERR_INVALID_ARG, "too many edges");
    const bool ci_dev = nnz > 0 && is_device_ptr(col_idx);
    if (flags & CC_VALIDATE) {
        std::vector<int32_t> hci;
        const int32_t *p = col_idx;
        if (ci_dev) {
            hci.resize(nnz);
            CC_CUDA(cudaMemcpy(hci.data(), col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
            p = hci.data();
        }
        CC_TRY(validate_host(n, rp.data(), p));
    }
    // member graph of every input vertex; no edge may join two members (each
    // member's count would otherwise take maps that reach into another)
    std::vector<int32_t> member_of;
    if (n_members > 1) {
        member_of.resize(n);
        for (int32_t i = 0; i < n_members; i++)
            for (int64_t v = moff[i]; v < moff[i + 1]; v++) member_of[v] = i;
        std::vector<int32_t> hci;
        const int32_t *p = col_idx;
        if (ci_dev) {
            hci.resize(nnz);
            CC_CUDA(cudaMemcpy(hci.data(), col_idx, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
            p = hci.data();
        }
        for (int64_t v = 0; v < n; v++)
            for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
                if (p[e] < 0 || p[e] >= n)
                    return fail(CC_ERR_BAD_GRAPH, "neighbour id out of range at vertex " + std::to_string(v));
                if (member_of[p[e]] != member_of[v])
                    return fail(CC_ERR_BAD_GRAPH, "edge " + std::to_string(v) + "-" + std::to_string(p[e]) +
                                                      " joins two member graphs");
            }
    }
    // Compact numbering: isolated vertices are dropped (they are in no embedding
    // when k >= 2).  By default the active vertices are also ordered by
    // decreasing degree, so the rows of the hub vertices -- the rows read most
    // often by the gathers -- sit together at the start of every table.
    // Graph batches keep each member's compact ids together (members in
    // input order, each ordered by degree), so every member's root rows form
    // one range.
    const bool by_degree = c->opt.vertex_order == 0;
    std::vector<int64_t> orig;
    g->n_members = n_members;
    g->h_member_off = moff;
    g->h_member_act.assign(n_members + 1, 0);
    for (int32_t i = 0; i < n_members; i++) {
        const size_t first = orig.size();
        for (int64_t v = moff[i]; v < moff[i + 1]; v++)
            if (rp[v + 1] > rp[v]) orig.push_back(v);
        if (by_degree)
            std::stable_sort(orig.begin() + first, orig.end(),
                             [&](int64_t x, int64_t y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
        g->h_member_act[i + 1] = (int64_t)orig.size();
    }
    g->h_new_id.assign(n, -1);
    g->h_row_ptr.assign(orig.size() + 1, 0);
    for (size_t i = 0; i < orig.size(); i++) {
        const int64_t v = orig[i], d = rp[v + 1] - rp[v];
        g->h_new_id[v] = (int32_t)i;
        g->h_row_ptr[i + 1] = g->h_row_ptr[i] + d;
        g->max_degree = std::max(g->max_degree, d);
    }
    g->n_act = (int64_t)orig.size();
    g->nnz = nnz;

    auto A = [&](uint64_t bytes) { return arena_alloc(c, bytes); };
    g->row_ptr = (int64_t *)A(sizeof(int64_t) * (g->n_act + 1));
    g->col_idx = (int32_t *)A(sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    g->orig = (int64_t *)A(sizeof(int64_t) * std::max<int64_t>(g->n_act, 1));
    g->member_act = (int64_t *)A(sizeof(int64_t) * (n_members + 1));
    int32_t *d_new = (int32_t *)A(sizeof(int32_t) * std::max<int64_t>(n, 1));
    int32_t *d_src = nullptr;
    int64_t *d_old_rp = nullptr;
    if (nnz > 0 && !ci_dev) d_src = (int32_t *)A(sizeof(int32_t) * nnz);
    if (nnz > 0 && by_degree) d_old_rp = (int64_t *)A(sizeof(int64_t) * (n + 1));
    if (!g->row_ptr || !g->col_idx || !g->orig || !g->member_act || !d_new || (nnz > 0 && !ci_dev && !d_src) ||
        (nnz > 0 && by_degree && !d_old_rp)) {
        c->arena.free(g->row_ptr);
        c->arena.free(g->col_idx);
        c->arena.free(g->orig);
        c->arena.free(g->member_act);
        c->arena.free(d_new);
        c->arena.free(d_src);
        c->arena.free(d_old_rp);
        return fail(CC_ERR_BUDGET, "graph does not fit the HBM budget");
    }
    CC_CUDA(cudaMemcpyAsync(g->row_ptr, g->h_row_ptr.data(), sizeof(int64_t) * (g->n_act + 1),
                            cudaMemcpyHostToDevice, st));
    CC_CUDA(cudaMemcpyAsync(g->orig, orig.data(), sizeof(int64_t) * g->n_act, cudaMemcpyHostToDevice, st));
    CC_CUDA(cudaMemcpyAsync(d_new, g->h_new_id.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    if (nnz > 0) {
        const int32_t *src = col_idx;
        if (!ci_dev) {
            CC_CUDA(cudaMemcpyAsync(d_src, col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
            src = d_src;
        }
        if (by_degree) {
            CC_CUDA(cudaMemcpyAsync(d_old_rp, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
            launch_permute_lists(st, g->n_act, n, g->orig, d_old_rp, g->row_ptr, src, d_new, g->col_idx);
        } else {
            // input order: isolated vertices hold no edges, so list offsets are unchanged
            launch_remap(st, nnz, n, src, d_new, g->col_idx);
        }
        c->launches++;
    }
    CC_CUDA(cudaMemcpyAsync(g->member_act, g->h_member_act.data(), sizeof(int64_t) * (n_members + 1),
                            cudaMemcpyHostToDevice, st));
    if (n_members > 1) {
        // colours are drawn from each vertex's id within its member graph, so a
        // member gets the colourings it would get loaded alone
        std::vector<int64_t> local(orig.size());
        for (size_t i = 0; i < orig.size(); i++) local[i] = orig[i] - moff[member_of[orig[i]]];
        CC_CUDA(cudaStreamSynchronize(st));  // the lists were permuted with the input ids
        CC_CUDA(cudaMemcpyAsync(g->orig, local.data(), sizeof(int64_t) * g->n_act, cudaMemcpyHostToDevice, st));
        CC_CUDA(cudaStreamSynchronize(st));
    }
    CC_CUDA(cudaGetLastError());
    CC_CUDA(cudaStreamSynchronize(st));
    c->arena.free(d_new);
    c->arena.free(d_src);
    c->arena.free(d_old_rp);
    int64_t id = c->next_id++;
    c->graphs[id] = std::move(g);
    *out = id;
    return CC_OK;
}

cc_status graph_free(Ctx *c, Graph *g)
{
    c->arena.free(g->row_ptr);
    c->arena.free(g->col_idx);
    c->arena.free(g->orig);
    c->arena.free(g->member_act);
    g->member_act = nullptr;
    c->arena.free(g->labels);
    g->labels = nullptr;
    for (auto &kv : g->splits) {
        c->arena.free(kv.second.heavy_v);
        c->arena.free(kv.second.heavy_tptr);
        c->arena.free(kv.second.task_e);
    }
    g->splits.clear();
    return CC_OK;
}

// Algorithm 4 (neighbour-list partitioning): a vertex whose list is longer than
// s gets ceil(deg / s) tasks of at most s neighbours; the tasks of one vertex
// are contiguous so their partial rows are summed without atomics.
cc_status ensure_split(Ctx *c, Graph *g, int64_t s, cudaStream_t st)
{
    if (g->splits.count(s)) return CC_OK;
    Graph::Split sp;
    sp.s = s;
    std::vector<int64_t> te;
    sp.h_heavy_tptr.push_back(0);
    for (int64_t v = 0; v < g->n_act; v++) {
        int64_t e0 = g->h_row_ptr[v], e1 = g->h_row_ptr[v + 1];
        if (e1 - e0 <= s) continue;
        sp.h_heavy_v.push_back((int32_t)v);
        for (int64_t e = e0; e < e1; e += s) {
            te.push_back(e);
            te.push_back(std::min(e + s, e1));
        }
        sp.h_heavy_tptr.push_back((int64_t)te.size() / 2);
    }
    sp.H = (int64_t)sp.h_heavy_v.size();
    sp.T = (int64_t)te.size() / 2;
    sp.heavy_v = (int32_t *)arena_alloc(c, sizeof(int32_t) * std::max<int64_t>(sp.H, 1));
    sp.heavy_tptr = (int64_t *)arena_alloc(c, sizeof(int64_t) * (sp.H + 1));
    sp.task_e = (int64_t *)arena_alloc(c, sizeof(int64_t) * std::max<int64_t>(2 * sp.T, 2));
    if (!sp.heavy_v || !sp.heavy_tptr || !sp.task_e) {
        c->arena.free(sp.heavy_v);
        c->arena.free(sp.heavy_tptr);
        c->arena.free(sp.task_e);
        return fail(CC_ERR_BUDGET, "task lists do not fit the HBM budget");
    }
    if (sp.H) {
        CC_CUDA(cudaMemcpyAsync(sp.heavy_v, sp.h_heavy_v.data(), sizeof(int32_t) * sp.H, cudaMemcpyHostToDevice, st));
        CC_CUDA(cudaMemcpyAsync(sp.task_e, te.data(), sizeof(int64_t) * te.size(), cudaMemcpyHostToDevice, st));
    }
    CC_CUDA(cudaMemcpyAsync(sp.heavy_tptr, sp.h_heavy_tptr.data(), sizeof(int64_t) * (sp.H + 1),
                            cudaMemcpyHostToDevice, st));
    CC_CUDA(cudaStreamSynchronize(st));
    g->splits[s] = std::move(sp);
    return CC_OK;
}

// Standalone table gather (cc_table_gather): the light / task / reduce kernels of
// the counting path on caller-provided device rows, task list and partial rows
// in the arena.
cc_status table_gather(Ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X,
                       uint64_t *agg, int64_t values, int32_t limbs, int32_t split)
{
    if (n < 0 || n >= (int64_t(1) << 31) || values < 1 || limbs < 1 || limbs > 4 || split < 0)
        return fail(CC_ERR_INVALID_ARG, "bad n, values, limbs or split_threshold");
    if (n == 0) return CC_OK;
    if (!row_ptr || !col_idx || !X || !agg) return fail(CC_ERR_INVALID_ARG, "NULL device pointer");
    const int64_t s = split > 0 ? split : 1024;
    cudaStream_t st = c->stream;
    std::vector<int64_t> rp(n + 1);
    CC_CUDA(cudaMemcpyAsync(rp.data(), row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    CC_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> hv;
    std::vector<int64_t> tptr{0}, te;
    for (int64_t v = 0; v < n; v++) {
        int64_t e0 = rp[v], e1 = rp[v + 1];
        if (e1 < e0) return fail(CC_ERR_INVALID_ARG, "row_ptr decreases");
        if (e1 - e0 <= s) continue;
        hv.push_back((int32_t)v);
        for (int64_t e = e0; e < e1; e += s) {
            te.push_back(e);
            te.push_back(std::min(e + s, e1));
        }
        tptr.push_back((int64_t)te.size() / 2);
    }
    const int64_t H = (int64_t)hv.size(), T = (int64_t)te.size() / 2;
    const uint64_t row_bytes = (uint64_t)values * limbs * 8;
    int32_t *d_hv = nullptr;
    int64_t *d_tptr = nullptr, *d_te = nullptr;
    uint64_t *d_part = nullptr;
    if (T > 0) {
        d_hv = (int32_t *)c->arena.alloc(sizeof(int32_t) * H);
        d_tptr = (int64_t *)c->arena.alloc(sizeof(int64_t) * (H + 1));
        d_te = (int64_t *)c->arena.alloc(sizeof(int64_t) * 2 * T);
        d_part = (uint64_t *)c->arena.alloc(row_bytes * T);
        if (!d_hv || !d_tptr || !d_te || !d_part) {
            c->arena.free(d_hv);
            c->arena.free(d_tptr);
            c->arena.free(d_te);
            c->arena.free(d_part);
            return fail(CC_ERR_BUDGET, "task scratch does not fit the arena");
        }
        CC_CUDA(cudaMemcpyAsync(d_hv, hv.data(), sizeof(int32_t) * H, cudaMemcpyHostToDevice, st));
        CC_CUDA(cudaMemcpyAsync(d_tptr, tptr.data(), sizeof(int64_t) * (H + 1), cudaMemcpyHostToDevice, st));
        CC_CUDA(cudaMemcpyAsync(d_te, te.data(), sizeof(int64_t) * 2 * T, cudaMemcpyHostToDevice, st));
    }
    launch_gather_light(st, limbs, limbs, 0, n, s, row_ptr, col_idx, X, values, agg);
    c->launches++;
    if (T > 0) {
        launch_gather_tasks(st, limbs, limbs, 0, T, col_idx, d_te, X, values, d_part);
        launch_gather_reduce(st, limbs, 0, H, 0, 0, d_hv, d_tptr, d_part, values, agg);
        c->launches += 2;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    c->arena.free(d_hv);
    c->arena.free(d_tptr);
    c->arena.free(d_te);
    c->arena.free(d_part);
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, std::string("table gather: ") + cudaGetErrorString(e));
    return CC_OK;
}

}  // namespace cc
