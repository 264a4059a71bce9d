// exec.cpp -- planning a template against a graph (integer widths, batch size,
// vertex blocks, static workspace layout) and running the per-colouring DP
// schedule (Algorithm 1's inner loop) as a sequence of kernel launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "runtime.h"

namespace cc {

uint64_t splitmix64_host(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

namespace {

constexpr uint64_t kAl = 256;
constexpr int kWorkCounters = 4096;  // per-pass work counters of the persistent gathers
inline uint64_t rup(uint64_t x) { return (x + kAl - 1) / kAl * kAl; }

int bits_for(double v)
{
    if (!(v >= 1.0)) return 1;
    // v is an upper bound computed in FP64; widen by a relative 1e-9 before taking bits
    return (int)std::floor(std::log2(v * (1.0 + 1e-9))) + 1;
}

// Rooted homomorphism counts (no colours): H_x(v) = prod over children c of
// sum_{u in N(v)} H_c(u), H_leaf = 1.  Every table entry X_x[v][S] counts a
// subset of these maps, so max_v H_x bounds the table and sum_v H_root bounds
// the total.
int bits_from_log2(double l2) { return l2 < 0 ? 1 : bits_for(std::exp2(std::min(l2, 1000.0))); }

// cache key of a chain's bounds: its rooted form and its steps' children
static std::string hom_key(const TemplatePlan &tp, int i)
{
    std::string key = tp.chains[i].canon + "|";
    for (auto &s : tp.chains[i].steps) key += (s.src_chain < 0 ? std::string("()") : tp.chains[s.src_chain].canon) + ";";
    return key;
}

cc_status hom_bounds(Ctx *c, Graph *g, const TemplatePlan &tp, cudaStream_t st, std::vector<double> *log2max,
                     double *log2sum_root, std::vector<std::vector<std::pair<double, double>>> *step_log2)
{
    const int nc = (int)tp.chains.size();
    log2max->assign(nc, 0.0);
    bool all = true;
    for (int i = 0; i < nc; i++)
        if (g->hom_cache.find(hom_key(tp, i)) == g->hom_cache.end()) all = false;
    if (!all) {
        int nsteps = 0;
        for (auto &C : tp.chains) nsteps += (int)C.steps.size();
        std::vector<double *> H(nc, nullptr);
        double *F = (double *)arena_alloc(c, sizeof(double) * std::max<int64_t>(g->n_act, 1));
        double *red = (double *)arena_alloc(c, 32 * (size_t)(nsteps + nc));
        bool ok = F && red;
        for (int i = 0; i < nc && ok; i++) {
            H[i] = (double *)arena_alloc(c, sizeof(double) * std::max<int64_t>(g->n_act, 1));
            ok = H[i] != nullptr;
        }
        if (!ok) {
            for (auto p : H) c->arena.free(p);
            c->arena.free(F);
            c->arena.free(red);
            return fail(CC_ERR_BUDGET, "no room for the homomorphism bound vectors");
        }
        // per step: (max, sum) of the bound after it and of its factor
        CC_CUDA(cudaMemsetAsync(red, 0, 32 * (size_t)(nsteps + nc), st));
        int q = 0;
        for (int i = 0; i < nc; i++) {
            launch_fill_double(st, g->n_act, 1.0, H[i]);
            for (auto &s : tp.chains[i].steps) {
                launch_hom_step(st, g->n_act, g->row_ptr, g->col_idx, s.src_chain < 0 ? nullptr : H[s.src_chain],
                                H[i], F);
                launch_max_sum(st, g->n_act, H[i], red + 4 * q);
                launch_max_sum(st, g->n_act, F, red + 4 * q + 2);
                q++;
            }
            c->launches += 1 + 3 * (int64_t)tp.chains[i].steps.size();
        }
        std::vector<double> h(4 * (size_t)q);
        CC_CUDA(cudaMemcpyAsync(h.data(), red, 32 * (size_t)q, cudaMemcpyDeviceToHost, st));
        CC_CUDA(cudaStreamSynchronize(st));
        auto l2 = [](double x) { return x > 0 ? std::log2(x) : -1.0; };
        q = 0;
        for (int i = 0; i < nc; i++) {
            Graph::HomBound hb;
            for (size_t si = 0; si < tp.chains[i].steps.size(); si++, q++) {
                hb.steps.push_back({l2(h[4 * q]), l2(h[4 * q + 2])});
                hb.l2max = l2(h[4 * q]);
                hb.l2sum = l2(h[4 * q + 1]);
            }
            g->hom_cache[hom_key(tp, i)] = hb;
        }
        CC_CUDA(cudaGetLastError());
        for (auto p : H) c->arena.free(p);
        c->arena.free(F);
        c->arena.free(red);
    }
    if (step_log2) step_log2->assign(nc, {});
    for (int i = 0; i < nc; i++) {
        const auto &hb = g->hom_cache[hom_key(tp, i)];
        (*log2max)[i] = hb.l2max;
        if (step_log2) (*step_log2)[i] = hb.steps;
    }
    *log2sum_root = g->hom_cache[hom_key(tp, nc - 1)].l2sum;
    return CC_OK;
}

// Limbs of every step's output and aggregate.  A step's values (colourful
// maps of the partial subtree) are bounded by its homomorphism bound, its
// aggregate by the step's factor sum_{u in N(v)} H_child(u); a step computes
// exactly at the smallest width above its bound, or modulo 2^(64 chain_L) when
// the bound exceeds the chain's width (which the ring maps to narrower widths
// preserve).  Widths never decrease along a chain; the last step writes the
// table at chain_L; an a = 1 step's output is its aggregate; a reused
// aggregate keeps the width it was computed at.
static cc_status step_widths(Ctx *c, Graph *g, PlanInstance *p, int width_bits, cudaStream_t st)
{
    const TemplatePlan &tp = p->tp;
    const int nc = (int)tp.chains.size();
    p->step_L.assign(nc, {});
    p->agg_L.assign(nc, {});
    std::vector<std::vector<std::pair<double, double>>> sl;
    if (width_bits == 0 && tp.k >= 2 && g->n_act > 0) {
        std::vector<double> l2max;
        double l2sum;
        CC_TRY(hom_bounds(c, g, tp, st, &l2max, &l2sum, &sl));
    }
    auto limbs = [](double l2) { return (bits_from_log2(l2) + 63) / 64; };
    for (int i = 0; i < nc; i++) {
        const auto &C = tp.chains[i];
        const int Lc = p->chain_L[i], n = (int)C.steps.size();
        auto &SL = p->step_L[i];
        auto &AL = p->agg_L[i];
        SL.assign(n, Lc);
        AL.assign(n, Lc);
        if (sl.empty() || (int)sl[i].size() != n) continue;  // fixed width: every step at the chain's
        for (int si = 0; si < n; si++) {
            int L = si + 1 == n ? Lc : std::min(Lc, limbs(sl[i][si].first));
            if (si > 0) L = std::max(L, SL[si - 1]);
            int A = std::min(L, std::min(Lc, limbs(sl[i][si].second)));
            if (C.steps[si].a == 1) A = L;
            if (C.steps[si].reuse_agg && si > 0) A = AL[si - 1];
            SL[si] = L;
            AL[si] = std::min(A, L);
        }
    }
    return CC_OK;
}

// consecutive vertices per work item of a column-segmented gather (fewer
// claims on the work counter when every row is split into segments)
static int vertex_group(int nch) { return nch > 1 ? 4 : 1; }

// Split of the light vertices of a block [v0, v1) for the fused kernels:
// [v0, vmid) with *nch column segments, [vmid, v1) whole rows.  Whole rows
// unless col_chunks > 0 asks for segments: their items are mostly low-degree
// vertices, for which every segment repeats the row-pointer -> neighbour-id
// -> row chain of dependent loads, and a chain's leaf steps then need a kernel
// of their own (R-MAT s22 / tree-12, two steps: whole rows 8.2 s; every light
// vertex segmented 9.5 s; only those of degree >= 64 segmented 8.55 s).
static int64_t fused_split(int col_chunks, int64_t v0, int64_t v1, int64_t R, int Ls, int *nch)
{
    *nch = col_chunks > 0 ? column_segments(R, Ls, col_chunks) : 1;
    return *nch > 1 ? v1 : v0;
}


struct Layout {
    uint64_t bytes = 0;
    uint64_t off_col, off_hist, off_act[2], off_agg, off_partial, off_root, off_scratch, off_totals, off_params,
        off_err, off_ctr, off_ncol = ~0ull;
    std::vector<uint64_t> off_table;
    int64_t max_tasks = 0;
    std::vector<std::pair<int64_t, int64_t>> blocks;
    std::vector<PlanInstance::BlockHeavy> heavy;
};

// Static workspace layout for batch B and block size V.  Count tables are
// placed first-fit over their lifetimes (a table lives from its chain to its
// last consumer), so memory is reused as soon as the schedule is done with it.
// keep_all: every table keeps its own memory for the whole pass (no reuse; the
// size a schedule without freeing needs, reported beside the real one).
Layout layout_for(const PlanInstance &p, const Graph &g, const Graph::Split &sp, int B, int64_t V,
                  bool keep_all = false)
{
    const TemplatePlan &tp = p.tp;
    const int k = tp.k;
    Layout Lo;
    const int64_t n = g.n_act;
    // blocks and their heavy ranges
    for (int64_t v0 = 0; v0 < n; v0 += V) Lo.blocks.push_back({v0, std::min(n, v0 + V)});
    for (auto &b : Lo.blocks) {
        PlanInstance::BlockHeavy h;
        h.h0 = std::lower_bound(sp.h_heavy_v.begin(), sp.h_heavy_v.end(), (int32_t)b.first) - sp.h_heavy_v.begin();
        h.h1 = std::lower_bound(sp.h_heavy_v.begin(), sp.h_heavy_v.end(), (int32_t)b.second) - sp.h_heavy_v.begin();
        h.t0 = sp.h_heavy_tptr[h.h0];
        h.t1 = sp.h_heavy_tptr[h.h1];
        h.edges = 0;
        for (int64_t i = h.h0; i < h.h1; i++) {
            const int32_t v = sp.h_heavy_v[i];
            h.edges += g.h_row_ptr[v + 1] - g.h_row_ptr[v];
        }
        Lo.max_tasks = std::max(Lo.max_tasks, h.t1 - h.t0);
        Lo.heavy.push_back(h);
    }
    // per-chain table sizes and lifetimes
    const int nc = (int)tp.chains.size();
    Lo.off_table.assign(nc, ~0ull);
    struct Placed { uint64_t off, size; int start, end; };
    std::vector<Placed> placed;
    uint64_t top = 0;
    for (int i = 0; i < nc; i++) {
        const auto &C = tp.chains[i];
        if (C.is_root) continue;
        uint64_t sz = rup((uint64_t)n * B * col_stride(binom(k, C.size)) * 8 * p.chain_L[i]);
        int start = i, end = keep_all ? nc : C.last_consumer;
        // lowest offset not overlapping any live placed table
        std::vector<std::pair<uint64_t, uint64_t>> busy;
        for (auto &q : placed)
            if (!(q.end < start || q.start > end)) busy.push_back({q.off, q.off + q.size});
        std::sort(busy.begin(), busy.end());
        uint64_t off = 0;
        for (auto &b : busy) {
            if (off + sz <= b.first) break;
            off = std::max(off, b.second);
        }
        placed.push_back({off, sz, start, end});
        Lo.off_table[i] = off;
        top = std::max(top, off + sz);
    }
    uint64_t cur = top;
    auto take = [&](uint64_t bytes) {
        uint64_t o = cur;
        cur += rup(bytes);
        return o;
    };
    // widest intermediate and aggregate rows
    int64_t maxAct = 1, maxP = 1;
    bool need_hist = false;
    for (auto &C : tp.chains)
        for (size_t si = 0; si < C.steps.size(); si++) {
            const auto &s = C.steps[si];
            if (si + 1 < C.steps.size()) maxAct = std::max<int64_t>(maxAct, col_stride(binom(k, s.h)));
            if (s.src_chain >= 0) maxP = std::max<int64_t>(maxP, col_stride(binom(k, s.p)));
            else need_hist = true;
        }
    const int Lm = p.Lmax;
    Lo.off_col = take((uint64_t)n * B);
    // neighbour colours of a one-colouring pass (AbsentSkip): one byte per list entry
    if (p.absent_skip && B == 1 && g.nnz > 0) Lo.off_ncol = take((uint64_t)g.nnz);
    Lo.off_hist = need_hist ? take((uint64_t)n * B * k * 4 * std::max<size_t>(1, p.hist_labels.size())) : 0;
    Lo.off_act[0] = take((uint64_t)V * B * maxAct * 8 * Lm);
    Lo.off_act[1] = take((uint64_t)V * B * maxAct * 8 * Lm);
    Lo.off_agg = take((uint64_t)V * B * maxP * 8 * Lm);
    Lo.off_partial = take((uint64_t)std::max<int64_t>(Lo.max_tasks, 1) * B * maxP * 8 * Lm);
    Lo.off_root = take((uint64_t)V * B * 8 * p.L_root);
    Lo.off_scratch = take((uint64_t)reduce_scratch_ctas() * B * 8 * p.L_root);
    Lo.off_totals = take((uint64_t)p.n_slots * p.n_members * B * 8 * p.L_root);
    Lo.off_params = take(sizeof(ColourParams));
    Lo.off_err = take(256);
    Lo.off_ctr = take(kWorkCounters * 8);
    Lo.bytes = cur;
    return Lo;
}

}  // namespace

namespace {

// The partition of one template against graph g: from its requested root, or
// the planner's choice (least modelled time with the widths each root needs),
// with every chain's integer width.
cc_status select_partition(Ctx *c, Graph *g, const Template *t, int width_bits, cudaStream_t st,
                           TemplatePlan *tp_out, std::vector<int> *chain_L_out, int *L_root_out)
{
    std::string err;
    const uint8_t *labels = t->labels.empty() ? nullptr : t->labels.data();
    if (labels && g->h_labels.empty())
        return fail(CC_ERR_INVALID_ARG, "labelled template on a graph without vertex labels");
    double avg = g->n_act ? (double)g->nnz / g->n_act : 1.0;
    // Integer widths of a partition: every chain at the smallest L with
    // max_v H(v) < 2^(64 L), capped at the root's L (which covers sum_v H).
    auto widths = [&](const TemplatePlan &tp, std::vector<int> *chain_L, int *L_root) -> cc_status {
        const int nc = (int)tp.chains.size();
        chain_L->assign(nc, 1);
        *L_root = 1;
        if (tp.k < 2 || g->n_act == 0) return CC_OK;
        if (width_bits != 0) {
            *L_root = width_bits / 64;
            for (auto &L : *chain_L) L = *L_root;
            return CC_OK;
        }
        std::vector<double> l2max;
        double l2sum;
        CC_TRY(hom_bounds(c, g, tp, st, &l2max, &l2sum, nullptr));
        const int rb = bits_from_log2(l2sum);
        if (rb > 256)
            return fail(CC_ERR_WIDTH, "exact counts may need " + std::to_string(rb) +
                                          " bits (> 256); request a fixed width_bits for residues");
        *L_root = (rb + 63) / 64;
        for (int i = 0; i < nc; i++) {
            const int b = bits_from_log2(l2max[i]);
            (*chain_L)[i] = tp.chains[i].is_root ? *L_root : std::min(*L_root, (b + 63) / 64);
        }
        return CC_OK;
    };
    // modelled time of a partition: bytes of its gathers and table writes at
    // their widths over HBM, plus its combine work (a multiply-add costs ~L^2)
    auto model = [&](const TemplatePlan &tp, const std::vector<int> &chain_L) {
        const double nnz = (double)g->nnz, na = (double)g->n_act;
        double bytes = 0, work = 0;
        for (size_t i = 0; i < tp.chains.size(); i++) {
            const auto &C = tp.chains[i];
            const double L = chain_L[i];
            if (!C.is_root) bytes += na * (double)col_stride(binom(tp.k, C.size)) * 8.0 * L;
            for (auto &s : C.steps) {
                if (s.src_chain >= 0 && !s.reuse_agg)
                    bytes += nnz * (double)col_stride(binom(tp.k, s.p)) * 8.0 * chain_L[s.src_chain];
                const double pr = s.a == 1 ? (double)binom(tp.k, s.h)
                                           : (double)binom(tp.k, s.h) * (double)binom(s.h, s.a);
                work += na * pr * L * L;
            }
        }
        return bytes / 6.0e12 + work / 3.0e11;
    };
    if (t->root_req >= 0 || t->k <= 2 || g->n_act == 0) {
        int rc = build_template_plan(t->k, t->edges.data(), t->root_req, 1, avg, &*tp_out, &err, labels);
        if (rc) return fail(rc, err);
        CC_TRY(widths(*tp_out, chain_L_out, L_root_out));
    } else {
        // the planner's root: the least modelled time with the widths each root
        // needs.  The model at 64-bit widths is a lower bound, so roots are tried
        // in its order and the search stops once that bound reaches the best.
        std::vector<std::pair<double, int>> rank;
        for (int r = 0; r < t->k; r++) {
            TemplatePlan tp;
            int rc = build_template_plan(t->k, t->edges.data(), r, 1, avg, &tp, &err, labels);
            if (rc) return fail(rc, err);
            rank.push_back({model(tp, std::vector<int>(tp.chains.size(), 1)), r});
        }
        std::sort(rank.begin(), rank.end());
        double best = 1e300;
        for (size_t ri = 0; ri < rank.size() && rank[ri].first < best; ri++) {
            const int r = rank[ri].second;
            TemplatePlan tp;
            int rc = build_template_plan(t->k, t->edges.data(), r, 1, avg, &tp, &err, labels);
            if (rc) return fail(rc, err);
            std::vector<int> cl;
            int lr = 1;
            CC_TRY(widths(tp, &cl, &lr));
            const double m = model(tp, cl);
            if (m < best) {
                best = m;
                *tp_out = tp;
                *chain_L_out = cl;
                *L_root_out = lr;
            }
        }
    }
    return CC_OK;
}

cc_status finish_plan(Ctx *c, Graph *g, PlanInstance *p, int n_iter, int width_bits, cudaStream_t st);

}  // namespace

cc_status make_plan(Ctx *c, int64_t gid, int64_t tid, int n_iter, int width_bits, cudaStream_t st,
                    std::unique_ptr<PlanInstance> *out, bool per_member)
{
    auto git = c->graphs.find(gid);
    if (git == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    auto tit = c->templates.find(tid);
    if (tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown template");
    if (width_bits != 0 && width_bits != 64 && width_bits != 128 && width_bits != 192 && width_bits != 256)
        return fail(CC_ERR_INVALID_ARG, "width_bits must be 0, 64, 128, 192 or 256");
    Graph *g = git->second.get();
    auto p = std::make_unique<PlanInstance>();
    p->graph_id = gid;
    p->tmpl_id = tid;
    CC_TRY(select_partition(c, g, tit->second.get(), width_bits, st, &p->tp, &p->chain_L, &p->L_root));
    const int nc = (int)p->tp.chains.size();
    p->n_slots = 1;
    p->n_members = per_member ? g->n_members : 1;
    p->chain_slot.assign(nc, -1);
    p->chain_slot[nc - 1] = 0;  // the root chain is last
    p->tmpl_slot = {0};
    p->tmpl_L = {p->L_root};
    p->tmpl_root = {p->tp.root};
    p->tmpl_aut = {p->tp.aut};
    CC_TRY(step_widths(c, g, p.get(), width_bits, st));
    CC_TRY(finish_plan(c, g, p.get(), n_iter, width_bits, st));
    *out = std::move(p);
    return CC_OK;
}

cc_status make_plan_multi(Ctx *c, int64_t gid, const std::vector<int64_t> &tids, int n_iter, int width_bits,
                          cudaStream_t st, std::unique_ptr<PlanInstance> *out)
{
    auto git = c->graphs.find(gid);
    if (git == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    if (tids.empty()) return fail(CC_ERR_INVALID_ARG, "no templates");
    if (width_bits != 0 && width_bits != 64 && width_bits != 128 && width_bits != 192 && width_bits != 256)
        return fail(CC_ERR_INVALID_ARG, "width_bits must be 0, 64, 128, 192 or 256");
    Graph *g = git->second.get();
    auto p = std::make_unique<PlanInstance>();
    p->graph_id = gid;
    p->tmpl_id = -1;
    TemplatePlan &M = p->tp;
    std::map<std::string, int> by_canon;  // rooted canonical form -> merged chain
    std::vector<int> Ls;
    p->n_slots = 0;
    p->L_root = 1;
    for (int64_t tid : tids) {
        auto tit = c->templates.find(tid);
        if (tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown template");
        const Template *t = tit->second.get();
        if (M.k == 0) M.k = t->k;
        if (t->k != M.k) return fail(CC_ERR_INVALID_ARG, "templates of one count must have the same k");
        TemplatePlan tp;
        std::vector<int> cl;
        int lr = 1;
        CC_TRY(select_partition(c, g, t, width_bits, st, &tp, &cl, &lr));
        p->sep_chains += (int)tp.chains.size();
        // chains in post-order; a chain whose rooted subtree is already planned
        // reuses that table (the table depends only on the rooted subtree)
        std::vector<int> map(tp.chains.size());
        for (size_t i = 0; i < tp.chains.size(); i++) {
            ChainPlan C = tp.chains[i];
            for (auto &st_ : C.steps)
                if (st_.src_chain >= 0 && !st_.reuse_agg)
                    p->sep_updates += (double)g->nnz * (double)binom(M.k, st_.p);
            auto it = by_canon.find(C.canon);
            if (it != by_canon.end()) {
                map[i] = it->second;
                Ls[it->second] = std::max(Ls[it->second], cl[i]);
                continue;
            }
            for (auto &st_ : C.steps)
                if (st_.src_chain >= 0) st_.src_chain = map[st_.src_chain];
            C.last_consumer = -1;
            map[i] = (int)M.chains.size();
            by_canon[C.canon] = map[i];
            M.chains.push_back(C);
            Ls.push_back(cl[i]);
            p->chain_slot.push_back(C.is_root ? p->n_slots++ : -1);
        }
        p->tmpl_slot.push_back(p->chain_slot[map.back()]);
        p->tmpl_L.push_back(lr);
        p->tmpl_root.push_back(tp.root);
        p->tmpl_aut.push_back(tp.aut);
        p->L_root = std::max(p->L_root, lr);
        M.table4_memory += tp.table4_memory;
        M.table4_computation += tp.table4_computation;
        M.pairs_per_vertex += tp.pairs_per_vertex;
    }
    M.root = p->tmpl_root[0];
    M.aut = 1;
    for (size_t ci = 0; ci < M.chains.size(); ci++)
        for (auto &st_ : M.chains[ci].steps)
            if (st_.src_chain >= 0) M.chains[st_.src_chain].last_consumer = (int)ci;
    // every root chain at the widest root width; template r keeps its low tmpl_L[r] limbs
    for (size_t ci = 0; ci < M.chains.size(); ci++)
        if (M.chains[ci].is_root) Ls[ci] = p->L_root;
    p->chain_L = Ls;
    CC_TRY(step_widths(c, g, p.get(), width_bits, st));
    CC_TRY(finish_plan(c, g, p.get(), n_iter, width_bits, st));
    *out = std::move(p);
    return CC_OK;
}

namespace {

// batch and block sizing under the budget, workspace layout, device constant
// tables and the analytic per-colouring figures of a selected partition
cc_status finish_plan(Ctx *c, Graph *g, PlanInstance *p, int n_iter, int width_bits, cudaStream_t st)
{
    const TemplatePlan &tp = p->tp;
    const int k = tp.k;
    const int nc = (int)tp.chains.size();
    p->hist_labels.clear();
    for (auto &C : tp.chains)
        for (auto &s : C.steps)
            if (s.src_chain < 0 &&
                std::find(p->hist_labels.begin(), p->hist_labels.end(), s.leaf_label) == p->hist_labels.end())
                p->hist_labels.push_back(s.leaf_label);
    p->width_bits = width_bits;
    p->exact = width_bits == 0;
    p->Lmax = *std::max_element(p->chain_L.begin(), p->chain_L.end());
    // gathers skip a neighbour's entries whose set lacks its colour (AbsentSkip):
    // colour masks fit 16 bits, ids 27 (the colour rides above them), and the
    // plan has a gathered table
    bool gathers = false;
    for (auto &C : tp.chains)
        for (auto &s : C.steps) gathers = gathers || s.src_chain >= 0;
    p->absent_skip = !c->opt.full_rows && k <= 16 && g->n_act < (int64_t(1) << 27) && gathers;
    // split threshold and batch / block size under the budget
    // default s = 4096: measured on R-MAT s22 / tree-12 (ms per step) 1024: 5590,
    // 2048: 5484, 4096: 5349, 8192: 5368, 16384: 5422, 65536: 6409 -- fewer
    // vertices on the task path save partial rows and per-vertex combines until
    // single warps on very long lists start to trail the launch
    int64_t split_default = 4096;
    int block_div = 1;
    p->col_chunks = c->opt.col_chunks;
    if (p->tmpl_id >= 0) {
        auto ts = c->tuned_shape.find({p->graph_id, p->tmpl_id});
        if (ts != c->tuned_shape.end()) {
            split_default = ts->second.split;
            if (c->opt.col_chunks == 0) p->col_chunks = ts->second.col_chunks;
            if (c->opt.block_vertices == 0) block_div = std::max(1, ts->second.block_div);
            p->shape_tuned = true;
        }
    }
    p->split = c->opt.split_threshold > 0 ? c->opt.split_threshold : split_default;
    CC_TRY(ensure_split(c, g, p->split, st));
    const Graph::Split &sp = g->splits[p->split];
    int Bmax = c->opt.batch > 0 ? c->opt.batch : 16;
    Bmax = std::max(1, std::min({Bmax, n_iter > 0 ? n_iter : 1, 64}));
    const uint64_t room = c->arena.largest_free();
    const int64_t n = std::max<int64_t>(g->n_act, 1);
    bool found = false;
    Layout Lo;
    for (int B = Bmax; B >= 1 && !found; B--) {
        int64_t V = c->opt.block_vertices > 0 ? std::min<int64_t>(c->opt.block_vertices, n) : n;
        while (true) {
            Lo = layout_for(*p, *g, sp, B, V);
            if (Lo.bytes + (64ull << 20) <= room) {
                found = true;
                if (block_div > 1 && V > 4096) {
                    // autotuned: a fraction of the largest block that fits (fits too)
                    V = std::max<int64_t>(4096, (V + block_div - 1) / block_div);
                    Lo = layout_for(*p, *g, sp, B, V);
                }
                p->B = B;
                p->V = V;
                break;
            }
            if (V <= 4096 || c->opt.block_vertices > 0) break;
            V = (V + 1) / 2;
        }
        if (c->opt.batch > 0 && !found) break;
    }
    if (!found) return fail(CC_ERR_BUDGET, "plan does not fit the HBM budget (largest free block " +
                                               std::to_string(room >> 20) + " MiB)");
    if (p->tmpl_id >= 0) {
        auto tm = c->tuned_modes.find(std::make_tuple(p->graph_id, p->tmpl_id, p->B));
        if (tm != c->tuned_modes.end()) {
            p->site_mode = tm->second;
            p->tuned = true;
        }
    }
    p->ws_bytes = Lo.bytes;
    // the same plan without freeing tables, without vertex blocking, and with
    // neither: the one-GPU counterparts of the paper's peak-memory comparison
    p->ws_no_reuse = layout_for(*p, *g, sp, p->B, p->V, true).bytes;
    p->ws_no_blocks = layout_for(*p, *g, sp, p->B, n).bytes;
    p->ws_naive = layout_for(*p, *g, sp, p->B, n, true).bytes;
    p->off_col = Lo.off_col;
    p->off_ncol = Lo.off_ncol;
    p->off_hist = Lo.off_hist;
    p->off_act[0] = Lo.off_act[0];
    p->off_act[1] = Lo.off_act[1];
    p->off_agg = Lo.off_agg;
    p->off_partial = Lo.off_partial;
    p->off_root = Lo.off_root;
    p->off_scratch = Lo.off_scratch;
    p->off_totals = Lo.off_totals;
    p->off_params = Lo.off_params;
    p->off_err = Lo.off_err;
    p->off_ctr = Lo.off_ctr;
    p->off_table = Lo.off_table;
    p->blocks = Lo.blocks;
    p->heavy = Lo.heavy;
    p->max_tasks = Lo.max_tasks;
    // device constants: rm tables (h = 1..k) and pair tables for generic steps
    SetTables T;
    T.build(k);
    std::vector<std::pair<int, int>> need_pairs;
    for (auto &C : tp.chains)
        for (auto &s : C.steps)
            if (s.a >= 2) need_pairs.push_back({s.h, s.a});  // p = 1 steps use the (h, h-1) table
    std::sort(need_pairs.begin(), need_pairs.end());
    need_pairs.erase(std::unique(need_pairs.begin(), need_pairs.end()), need_pairs.end());
    // per set size h: for each colour, the ranks of the h-sets holding it
    // (k * C(k-1, h-1) entries; k * 2^(k-1) over all h)
    std::map<int, std::vector<uint16_t>> elig;
    for (int h = 1; h <= k; h++) {
        std::vector<uint16_t> &el = elig[h];
        for (int cc = 0; cc < k; cc++)
            for (int64_t r = 0; r < binom(k, h); r++)
                if (T.mask_of_rank[h][r] >> cc & 1) el.push_back((uint16_t)r);
    }
    // per set size h: the colour mask of each column of a row (0 for the padding)
    std::vector<std::vector<uint16_t>> smask(k + 1);
    for (int h = 1; h <= k; h++) {
        smask[h].assign(col_stride(binom(k, h)), 0);
        for (int64_t r = 0; r < binom(k, h); r++) smask[h][r] = (uint16_t)T.mask_of_rank[h][r];
    }
    uint64_t cbytes = 0;
    for (int h = 1; h <= k; h++) cbytes += rup(smask[h].size() * 2);
    for (auto &kv : elig) cbytes += rup(kv.second.size() * 2);
    for (int h = 1; h <= k; h++) cbytes += rup(T.rm[h].size() * 2);
    for (int q = 0; q < k; q++) cbytes += rup(T.ad[q].size() * 2);
    std::vector<std::vector<uint32_t>> pt;
    for (auto &hp : need_pairs) {
        pt.push_back(T.pairs(hp.first, hp.second));
        cbytes += rup(pt.back().size() * 4);
    }
    p->consts = arena_alloc(c, std::max<uint64_t>(cbytes, 256));
    if (!p->consts) return fail(CC_ERR_BUDGET, "no room for colour-set tables");
    char *cp = (char *)p->consts;
    p->d_rm.assign(k + 1, nullptr);
    for (int h = 1; h <= k; h++) {
        p->d_rm[h] = (uint16_t *)cp;
        CC_CUDA(cudaMemcpyAsync(cp, T.rm[h].data(), T.rm[h].size() * 2, cudaMemcpyHostToDevice, st));
        cp += rup(T.rm[h].size() * 2);
    }
    p->d_ad.assign(k + 1, nullptr);
    for (int q = 0; q < k; q++) {
        p->d_ad[q] = (uint16_t *)cp;
        CC_CUDA(cudaMemcpyAsync(cp, T.ad[q].data(), T.ad[q].size() * 2, cudaMemcpyHostToDevice, st));
        cp += rup(T.ad[q].size() * 2);
    }
    p->d_smask.assign(k + 1, nullptr);
    for (int h = 1; h <= k; h++) {
        p->d_smask[h] = (uint16_t *)cp;
        CC_CUDA(cudaMemcpyAsync(cp, smask[h].data(), smask[h].size() * 2, cudaMemcpyHostToDevice, st));
        cp += rup(smask[h].size() * 2);
    }
    p->d_elig.clear();
    for (auto &kv : elig) {
        p->d_elig[kv.first] = (uint16_t *)cp;
        CC_CUDA(cudaMemcpyAsync(cp, kv.second.data(), kv.second.size() * 2, cudaMemcpyHostToDevice, st));
        cp += rup(kv.second.size() * 2);
    }
    for (size_t i = 0; i < need_pairs.size(); i++) {
        p->d_pairs[need_pairs[i]] = (uint32_t *)cp;
        CC_CUDA(cudaMemcpyAsync(cp, pt[i].data(), pt[i].size() * 4, cudaMemcpyHostToDevice, st));
        cp += rup(pt[i].size() * 4);
    }
    CC_CUDA(cudaStreamSynchronize(st));
    // analytic per-colouring figures
    const double nnz = (double)g->nnz, na = (double)g->n_act;
    int gather_passes = 0;
    for (int i = 0; i < nc; i++) {
        const auto &C = tp.chains[i];
        for (auto &s : C.steps) {
            double pairs_v = s.a == 1 ? (double)binom(k, s.h)
                                      : (s.p == 1 ? (double)binom(k, s.h) * s.h : (double)binom(k, s.h) * binom(s.h, s.a));
            p->pairs += na * pairs_v;
            // 64-bit limb multiplications of a general combine (a >= 2, gathered child) at its widths
            if (s.a >= 2 && s.src_chain >= 0) {
                const int L = p->step_L[i][&s - C.steps.data()];
                const int La = &s == C.steps.data() ? L : p->step_L[i][&s - C.steps.data() - 1];
                const int Lb = p->agg_L[i][&s - C.steps.data()];
                int m = 0;
                for (int x = 0; x < La; x++)
                    for (int y = 0; y < Lb && x + y < L; y++) m += 1 + (x + y + 1 < L);
                p->limb_products += na * pairs_v * m;
            }
            if (s.src_chain >= 0 && !s.reuse_agg) {
                double cols = (double)binom(k, s.p);
                p->updates += nnz * cols;
                p->gather_bytes += nnz * cols * 8.0 * p->chain_L[s.src_chain];
                gather_passes++;
            }
        }
        if (!C.is_root) p->alg_bytes += na * (double)binom(k, C.size) * 8.0 * p->chain_L[i];
    }
    p->alg_bytes += p->gather_bytes;
    p->alg_bytes += gather_passes * (4.0 * nnz + 8.0 * (na + 1)) / p->B;  // CSR, shared by the pass
    bool any_leaf = false;
    for (auto &C : tp.chains)
        for (auto &s : C.steps) any_leaf |= s.src_chain < 0;
    if (any_leaf) p->alg_bytes += nnz + (4.0 * nnz + 8.0 * (na + 1)) / p->B;  // colour bytes + CSR
    return CC_OK;
}

}  // namespace

void free_plan(Ctx *c, PlanInstance *p)
{
    if (!p) return;
    c->arena.free(p->consts);
    p->consts = nullptr;
}

namespace {

struct Launcher {
    Ctx *c;
    cudaStream_t st;
    KernelTimer &T;
    Launcher(Ctx *c_, cudaStream_t s) : c(c_), st(s), T(c_->timer) {}
    int kind = -1;
    cudaEvent_t ea = nullptr;
    cudaEvent_t get_event()
    {
        if (T.pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = T.pool.back();
        T.pool.pop_back();
        return e;
    }
    void begin(int k_)
    {
        kind = k_;
        take_launch_names();  // names noted outside a timed kind are dropped
        if (T.on) {
            ea = get_event();
            cudaEventRecord(ea, st);
        }
    }
    void end(int nlaunch, double bytes)
    {
        c->launches += nlaunch;
        // the instantiations this bracket launched; one alone gets its time
        std::string only;
        int64_t n_only = 0;
        for (auto &nm : take_launch_names()) {
            T.instances[kind][nm].launches++;
            if (n_only == 0 || nm == only) {
                only = nm;
                n_only++;
            } else {
                n_only = -1 << 30;
            }
        }
        if (n_only <= 0) only.clear();
        T.launches[kind] += nlaunch;
        T.total_launches += nlaunch;
        T.bytes[kind] += bytes;
        if (T.on) {
            cudaEvent_t eb = get_event();
            cudaEventRecord(eb, st);
            T.pending.push_back({ea, eb, kind, bytes, only, n_only});
        }
    }
};

}  // namespace

// Resolve pending event pairs into the per-kind totals (after a stream sync).
static void drain_timer(Ctx *c)
{
    auto &T = c->timer;
    for (auto &q : T.pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            T.seconds[q.kind] += ms * 1e-3;
            if (!q.only.empty()) {
                auto &in = T.instances[q.kind][q.only];
                in.seconds += ms * 1e-3;
                in.bytes += q.bytes;
                in.timed_launches += q.n;
            }
        }
        T.pool.push_back(q.a);
        T.pool.push_back(q.b);
    }
    cudaGetLastError();
    T.pending.clear();
}

// With cc_options.l2_persist_mb: the stream's L2 access window over the first
// bytes of a table about to be gathered, where degree ordering puts the rows
// read most often (hits persist in the set-aside L2, misses stream).  Not
// changed while the stream is being captured.
static void l2_window(Ctx *c, cudaStream_t st, const void *X, uint64_t table_bytes)
{
    if (c->l2_window_bytes == 0) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    cudaStreamAttrValue v{};
    v.accessPolicyWindow.base_ptr = const_cast<void *>(X);
    v.accessPolicyWindow.num_bytes = std::min<uint64_t>(c->l2_window_bytes, table_bytes);
    v.accessPolicyWindow.hitRatio = 1.0f;
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess) cudaGetLastError();
}

static cc_status launch_pass(Ctx *c, PlanInstance *p, char *ws, cudaStream_t st, const int64_t *d_samples,
                             int64_t n_samples, uint64_t *d_samples_out, bool tune = false)
{
    Graph *g = c->graphs.at(p->graph_id).get();
    const TemplatePlan &tp = p->tp;
    const int k = tp.k, B = p->B;
    const Graph::Split &sp = g->splits.at(p->split);
    Launcher Ln(c, st);
    auto W = [&](uint64_t off) { return ws + off; };
    uint64_t *totals = (uint64_t *)W(p->off_totals);
    CC_CUDA(cudaMemsetAsync(totals, 0, (size_t)p->totals_words() * 8, st));
    uint8_t *col = (uint8_t *)W(p->off_col);
    unsigned long long *ctr = (unsigned long long *)W(p->off_ctr);
    // Every persistent launch pulls its work items from a zeroed counter of its
    // own.  A pass with more launches than counters (many small vertex blocks)
    // clears them all again once they are used up: the clear is ordered on the
    // stream after every launch that used them.  (A failed clear is reported by
    // the cudaGetLastError at the end of the pass.)
    int ctr_used = 0;
    auto next_counter = [&]() -> unsigned long long * {
        if (ctr_used == kWorkCounters) {
            cudaMemsetAsync(ctr, 0, (size_t)kWorkCounters * 8, st);
            ctr_used = 0;
        }
        return ctr + ctr_used++;
    };
    CC_CUDA(cudaMemsetAsync(ctr, 0, (size_t)kWorkCounters * 8, st));
    Ln.begin(K_COLOUR);
    launch_colour(st, g->n_act, B, k, g->orig, (const ColourParams *)W(p->off_params), col);
    Ln.end(1, (double)g->n_act * (8 + B));
    // one colouring per pass: the gathers load only the entries of a neighbour's
    // row whose colour set holds the neighbour's colour (the rest are zero)
    const uint8_t *ncol = nullptr;
    if (p->off_ncol != ~0ull && B == 1) {
        Ln.begin(K_COLOUR);
        launch_neighbour_colours(st, g->nnz, g->col_idx, col, (uint8_t *)W(p->off_ncol));
        Ln.end(1, (double)g->nnz * 6);
        ncol = (const uint8_t *)W(p->off_ncol);
    }
    // the skip for gathering a table of sets of size h
    auto skip_for = [&](int h) {
        AbsentSkip sk;
        if (ncol) {
            sk.ncol = ncol;
            sk.smask = p->d_smask.at(h);
        }
        return sk;
    };
    uint32_t *hist = (uint32_t *)W(p->off_hist);
    // the histogram of a leaf child with label `lab` (-1: all neighbours)
    auto hist_for = [&](int lab) -> uint32_t * {
        for (size_t i = 0; i < p->hist_labels.size(); i++)
            if (p->hist_labels[i] == lab) return hist + i * (uint64_t)g->n_act * B * k;
        return hist;
    };
    if (!p->hist_labels.empty()) {
        Ln.begin(K_HIST);
        for (int lab : p->hist_labels)
            launch_hist(st, 0, g->n_act, B, k, g->row_ptr, g->col_idx, col, hist_for(lab),
                        lab >= 0 ? g->labels : nullptr, lab);
        Ln.end(1, (double)g->nnz * (4 + B) + (double)g->n_act * (8 + 4.0 * B * k));
    }
    if (p->step_path.size() != tp.chains.size()) {
        p->step_path.assign(tp.chains.size(), {});
        for (size_t ci = 0; ci < tp.chains.size(); ci++) p->step_path[ci].assign(tp.chains[ci].steps.size(), {});
    }
    for (size_t ci = 0; ci < tp.chains.size(); ci++) {
        const ChainPlan &C = tp.chains[ci];
        const int L = p->chain_L[ci];
        for (size_t bi = 0; bi < p->blocks.size(); bi++) {
            // the path of step si for the light vertices of the first block
            auto note_path = [&](size_t si, int path, int l0, int l1, int l2) {
                if (bi == 0) p->step_path[ci][si] = {path, l0, l1, l2};
            };
            const int64_t v0 = p->blocks[bi].first, v1 = p->blocks[bi].second, nv = v1 - v0;
            const auto &hv = p->heavy[bi];
            const uint64_t *cur = nullptr;
            int64_t cur_stride = k;
            uint64_t *root_rows = (uint64_t *)W(p->off_root);
            // output row block and stride of step si of this chain
            auto step_out = [&](size_t si, int64_t *Chs_out) -> uint64_t * {
                const bool last = si + 1 == C.steps.size();
                const int64_t Ch = binom(k, C.steps[si].h);
                // root rows hold one column and are never gathered: no padding
                const int64_t Chs = (last && C.is_root) ? 1 : col_stride(Ch);
                *Chs_out = Chs;
                if (last)
                    return C.is_root ? root_rows : (uint64_t *)W(p->off_table[ci]) + (uint64_t)v0 * B * Chs * L;
                return (uint64_t *)W(p->off_act[si & 1]);
            };
            // Chain fusion: a fused first step followed only by leaf (p = 1) steps
            // runs as one kernel for light vertices; heavy vertices (a prefix of the
            // block under degree ordering) take the task path and the p = 1 kernels.
            size_t nleaf = 0;
            if (c->opt.fused && c->opt.vertex_order == 0 && C.steps.size() >= 2 && C.steps[0].a == 1 &&
                C.steps[0].src_chain >= 0 && !C.steps[1].reuse_agg && C.steps.size() - 1 <= 15) {
                nleaf = C.steps.size() - 1;
                for (size_t j = 1; j < C.steps.size(); j++)
                    if (C.steps[j].src_chain >= 0) nleaf = 0;
                // heavy vertices of the block must be its first rows
                if (hv.h1 > hv.h0 && (sp.h_heavy_v[hv.h0] != v0 || sp.h_heavy_v[hv.h1 - 1] != v0 + (hv.h1 - hv.h0) - 1))
                    nleaf = 0;
            }
            if (nleaf > 0) {
                const Step &s = C.steps[0];
                const int Ls = p->chain_L[s.src_chain];
                const int64_t Cp = binom(k, s.p), Cps = col_stride(Cp);
                const int64_t R = (int64_t)B * Cps;
                const uint64_t *X = (const uint64_t *)W(p->off_table[s.src_chain]);
                l2_window(c, st, X, (uint64_t)g->n_act * R * Ls * 8);
                uint64_t *agg = (uint64_t *)W(p->off_agg);
                int64_t Chs0;
                uint64_t *out0 = step_out(0, &Chs0);
                const int64_t Ch0 = binom(k, s.h);
                // Intermediate steps alternate between the two act buffers with their
                // own row strides; inside one kernel a vertex's rows for step j + 2
                // would then land on other vertices' step-j rows, so every light
                // vertex gets one slot of the widest intermediate row instead.  The
                // last step writes the chain's table (its own buffer, usual stride).
                int64_t slot = 0;
                for (size_t j = 0; j < nleaf; j++) slot = std::max(slot, col_stride(binom(k, C.steps[j].h)));
                slot *= (int64_t)B * L;
                auto vstride = [&](size_t j, int64_t cs) { return j == nleaf ? (int64_t)B * cs * L : slot; };
                LeafChain lc{};
                lc.n = (int)nleaf;
                lc.col = col;
                for (size_t j = 1; j <= nleaf; j++) {
                    int64_t cs;
                    lc.out[j - 1] = step_out(j, &cs);
                    lc.h[j - 1] = C.steps[j].h;
                    lc.Ch[j - 1] = binom(k, C.steps[j].h);
                    lc.Chs[j - 1] = cs;
                    lc.vs[j - 1] = vstride(j, cs);
                    lc.pairs[j - 1] = p->d_pairs.at({C.steps[j].h, C.steps[j].a});
                    lc.rm[j - 1] = p->d_rm[C.steps[j].h];
                    lc.elig[j - 1] = p->d_elig.at(C.steps[j].h);
                    lc.E[j - 1] = (int)binom(k - 1, C.steps[j].h - 1);
                    lc.hist[j - 1] = hist_for(C.steps[j].leaf_label);
                }
                const int64_t nh = hv.h1 - hv.h0;
                // algorithmic bytes of the chain for `nvert` vertices with `edges` list entries:
                // neighbour rows + ids + row pointers + the step rows written, and per
                // leaf step the previous row and the colour histogram read
                auto chain_bytes = [&](double edges, double nvert) {
                    double b = edges * ((double)B * Cp * 8.0 * Ls + 4) + nvert * 8.0 + nvert * B * Ch0 * 8.0 * L;
                    for (size_t j = 1; j <= nleaf; j++)
                        b += nvert * B * ((binom(k, C.steps[j].h) + binom(k, C.steps[j].a)) * 8.0 * L + 4.0 * k);
                    return b;
                };
                const double e_blk = (double)(g->h_row_ptr[v1] - g->h_row_ptr[v0]);
                // [v0, vmid): column-segmented gather + select into the slots, then the
                // leaf kernel; [vmid, v1): the one-kernel chain (whole rows)
                int nch = 1;
                const int64_t vmid = fused_split(p->col_chunks, v0, v1, R, Ls, &nch);
                int nl = 0;
                // the fused step at its own width (at most one limb below the chain's)
                const int Lf = std::max(L - 1, std::min(L, p->step_L[ci][0]));
                note_path(0, vmid > v0 ? CC_PATH_SEGMENTED : CC_PATH_CHAIN_KERNEL, Ls, vmid > v0 ? L : Lf, L);
                for (size_t j = 1; j <= nleaf; j++) note_path(j, CC_PATH_IN_CHAIN, Ls, vmid > v0 ? L : Lf, L);
                Ln.begin(K_FUSED);
                if (vmid > v0) {
                    launch_gather_select(st, Ls, L, v0, vmid, p->split, g->row_ptr, g->col_idx, X, B, k, Cp, Cps, Ch0,
                                         Chs0, p->d_ad[s.p], p->d_rm[s.h], col, out0, next_counter(), 4, nch,
                                         vertex_group(nch), vstride(0, Chs0), skip_for(s.p));
                    launch_leaf_chain(st, L, v0, vmid, p->split, g->row_ptr, B, k, out0, vstride(0, Chs0), Chs0, lc,
                                      next_counter());
                    nl += 2;
                }
                if (v1 > vmid) {
                    // rows of vertex v stay at (v - v0) * stride: shift the outputs by vmid - v0
                    LeafChain lt = lc;
                    for (int j = 0; j < lt.n; j++) lt.out[j] += (vmid - v0) * lt.vs[j];
                    launch_gather_select_chain(st, Ls, Lf, L, vmid, v1, p->split, g->row_ptr, g->col_idx, X, B, k, Cp, Cps,
                                               Ch0, Chs0, p->d_ad[s.p], p->d_rm[s.h], col,
                                               out0 + (vmid - v0) * vstride(0, Chs0), vstride(0, Chs0), lt,
                                               next_counter(), 4, skip_for(s.p));
                    nl++;
                }
                Ln.end(nl, chain_bytes(e_blk - (double)hv.edges, (double)(nv - nh)));
                if (nh > 0) {
                    // heavy vertices (Algorithm 4): tasks, partial-row sums, select, leaf steps
                    Ln.begin(K_HEAVY);
                    uint64_t *part = (uint64_t *)W(p->off_partial);
                    launch_gather_tasks(st, Ls, L, hv.t0, hv.t1, g->col_idx, sp.task_e, X, R, part, false,
                                        next_counter(), 4, column_segments(R, Ls, p->col_chunks), skip_for(s.p));
                    launch_gather_reduce(st, L, hv.h0, hv.h1, v0, hv.t0, sp.heavy_v, sp.heavy_tptr, part, R, agg);
                    launch_select_heavy(st, L, hv.h0, hv.h1, v0, sp.heavy_v, B, k, Ch0, Chs0, Cps, p->d_rm[s.h], col,
                                        agg, out0);
                    const uint64_t *prev = out0;
                    int64_t prev_s = Chs0;
                    for (int j = 0; j < lc.n; j++) {
                        launch_combine_hist(st, L, L, nh, B, k, lc.Ch[j], lc.Chs[j], prev_s, lc.h[j], lc.pairs[j],
                                            prev, lc.hist[j] + (uint64_t)v0 * B * k, lc.out[j], col + (uint64_t)v0 * B,
                                            lc.rm[j], lc.elig[j], lc.E[j]);
                        prev = lc.out[j];
                        prev_s = lc.Chs[j];
                    }
                    Ln.end(3 + lc.n, chain_bytes((double)hv.edges, (double)nh));
                }
            }
            for (size_t si = nleaf > 0 ? C.steps.size() : 0; si < C.steps.size(); si++) {
                const Step &s = C.steps[si];
                const int64_t Ch = binom(k, s.h);
                int64_t Chs;
                uint64_t *out = step_out(si, &Chs);
                // limbs of this step's output, of the previous step's rows and of the aggregate
                const int Lo = p->step_L[ci][si], La = si > 0 ? p->step_L[ci][si - 1] : Lo, Lg = p->agg_L[ci][si];
                if (s.src_chain < 0) {
                    const uint32_t *hrow = hist_for(s.leaf_label) + (uint64_t)v0 * B * k;
                    if (s.a == 1) {
                        note_path(si, CC_PATH_LEAF_SELECT, 0, 0, Lo);
                        Ln.begin(K_SELECT);
                        launch_combine_select(st, Lo, true, v0, nv, B, k, Ch, Chs, k, p->d_rm[s.h], col, hrow, out);
                        Ln.end(1, (double)nv * B * (Ch * 8.0 * Lo + 4.0 * k + 1));
                    } else {
                        note_path(si, CC_PATH_LEAF_COMBINE, La, 0, Lo);
                        Ln.begin(K_CHIST);
                        launch_combine_hist(st, Lo, La, nv, B, k, Ch, Chs, cur_stride, s.h, p->d_pairs.at({s.h, s.a}),
                                            cur, hrow, out, col + (uint64_t)v0 * B, p->d_rm[s.h], p->d_elig.at(s.h),
                                            binom(k - 1, s.h - 1));
                        Ln.end(1, (double)nv * B * (Ch * 8.0 * Lo + binom(k, s.a) * 8.0 * La + 4.0 * k));
                    }
                } else if (c->opt.fused && s.a == 1 && !s.reuse_agg &&
                           !(si + 1 < C.steps.size() && C.steps[si + 1].reuse_agg)) {
                    // a3 + a4 fused: the aggregate of light vertices goes straight into out
                    const int Ls = p->chain_L[s.src_chain];
                    const int64_t Cp = binom(k, s.p), Cps = col_stride(Cp);
                    const int64_t R = (int64_t)B * Cps;
                    const uint64_t *X = (const uint64_t *)W(p->off_table[s.src_chain]);
                    l2_window(c, st, X, (uint64_t)g->n_act * R * Ls * 8);
                    uint64_t *agg = (uint64_t *)W(p->off_agg);
                    // algorithmic bytes: neighbour rows + ids + row pointers + output rows
                    auto sel_bytes = [&](double edges, double nvert) {
                        return edges * ((double)B * Cp * 8.0 * Ls + 4) + nvert * 8.0 + nvert * B * Ch * 8.0 * Lo;
                    };
                    const double e_blk = (double)(g->h_row_ptr[v1] - g->h_row_ptr[v0]);
                    const double light_bytes = sel_bytes(e_blk - (double)hv.edges, (double)(nv - (hv.h1 - hv.h0)));
                    note_path(si, CC_PATH_FUSED_SELECT, Ls, 0, Lo);
                    Ln.begin(K_FUSED);
                    const auto site = std::make_pair((int)ci, (int)si);
                    int nch = 1;
                    const int64_t vmid = fused_split(p->col_chunks, v0, v1, R, Ls, &nch);
                    // [v0, vmid) column-segmented, [vmid, v1) whole rows
                    auto fused_run = [&](int nb) {
                        if (vmid > v0)
                            launch_gather_select(st, Ls, Lo, v0, vmid, p->split, g->row_ptr, g->col_idx, X, B, k, Cp,
                                                 Cps, Ch, Chs, p->d_ad[s.p], p->d_rm[s.h], col, out, next_counter(),
                                                 nb, nch, vertex_group(nch), 0, skip_for(s.p));
                        if (v1 > vmid)
                            launch_gather_select(st, Ls, Lo, vmid, v1, p->split, g->row_ptr, g->col_idx, X, B, k, Cp,
                                                 Cps, Ch, Chs, p->d_ad[s.p], p->d_rm[s.h], col,
                                                 out + (vmid - v0) * B * Chs * Lo, next_counter(), nb, 1, 1, 0,
                                                 skip_for(s.p));
                    };
                    int nl = 0, nb_tasks = 2;
                    if (tune) {
                        for (int nb : {2, 4}) {  // the default (4) last
                            PlanInstance::Trial tr{(int)ci, (int)si, nb, nullptr, nullptr};
                            cudaEventCreate(&tr.a);
                            cudaEventCreate(&tr.b);
                            cudaEventRecord(tr.a, st);
                            fused_run(nb);
                            cudaEventRecord(tr.b, st);
                            p->trials.push_back(tr);
                            nl++;
                        }
                    } else {
                        auto it = p->site_mode.find(site);
                        nb_tasks = (it != p->site_mode.end() && it->second == 2) ? 2 : 4;
                        fused_run(nb_tasks);
                        nl = 1;
                    }
                    Ln.end(nl, nl * light_bytes);
                    if (hv.t1 > hv.t0) {
                        // heavy vertices (Algorithm 4): tasks, partial-row sums, select
                        Ln.begin(K_HEAVY);
                        uint64_t *part = (uint64_t *)W(p->off_partial);
                        launch_gather_tasks(st, Ls, Lo, hv.t0, hv.t1, g->col_idx, sp.task_e, X, R, part, false,
                                            next_counter(), nb_tasks, column_segments(R, Ls, p->col_chunks),
                                            skip_for(s.p));
                        launch_gather_reduce(st, Lo, hv.h0, hv.h1, v0, hv.t0, sp.heavy_v, sp.heavy_tptr, part, R, agg);
                        launch_select_heavy(st, Lo, hv.h0, hv.h1, v0, sp.heavy_v, B, k, Ch, Chs, Cps, p->d_rm[s.h], col,
                                            agg, out);
                        Ln.end(3, sel_bytes((double)hv.edges, (double)(hv.h1 - hv.h0)));
                    }
                } else {
                    const int Ls = p->chain_L[s.src_chain];
                    const int64_t Cp = binom(k, s.p), Cps = col_stride(Cp);
                    const int64_t R = (int64_t)B * Cps;
                    const uint64_t *X = (const uint64_t *)W(p->off_table[s.src_chain]);
                    l2_window(c, st, X, (uint64_t)g->n_act * R * Ls * 8);
                    uint64_t *agg = (uint64_t *)W(p->off_agg);
                    if (!s.reuse_agg) {
                        // algorithmic bytes of this gather: neighbour rows + CSR + aggregate write
                        auto g_bytes = [&](double edges, double nvert) {
                            return edges * ((double)B * Cp * 8.0 * Ls + 4) + nvert * 8.0 + nvert * B * Cp * 8.0 * Lg;
                        };
                        const double e_blk = (double)(g->h_row_ptr[v1] - g->h_row_ptr[v0]);
                        const int64_t nh = hv.h1 - hv.h0;
                        const double light_bytes = g_bytes(e_blk - (double)hv.edges, (double)(nv - nh));
                        const double heavy_bytes = g_bytes((double)hv.edges, (double)nh);
                        int *err = (int *)W(p->off_err);
                        // light vertices timed as "gather", heavy ones (Algorithm 4 tasks) as "heavy"
                        auto run_gather = [&](int gm) {
                            const bool bulk = gm == 0 && bulk_gather_ok(Ls, R);
                            const bool group = gm == 3 && vec_gather_ok(Ls, R);
                            const bool vec = !bulk && !group && (gm == 0 || gm == 2) && vec_gather_ok(Ls, R);
                            Ln.begin(K_GATHER);
                            if (bulk)
                                launch_gather_light_bulk(st, Ls, Lg, v0, v1, p->split, g->row_ptr, g->col_idx, g->nnz,
                                                         X, R, agg, err);
                            else if (group)
                                launch_gather_light_group(st, Ls, Lg, v0, v1, p->split, g->row_ptr, g->col_idx, X, R,
                                                          agg);
                            else if (vec)
                                launch_gather_light_vec(st, Ls, Lg, v0, v1, p->split, g->row_ptr, g->col_idx, X, R, agg);
                            else
                                launch_gather_light(st, Ls, Lg, v0, v1, p->split, g->row_ptr, g->col_idx, X, R, agg,
                                                    gm == 4, gm == 5 ? nullptr : next_counter(), gm == 6 ? 2 : 4,
                                                    column_segments(R, Ls, p->col_chunks),
                                                    vertex_group(column_segments(R, Ls, p->col_chunks)),
                                                    skip_for(s.p));
                            Ln.end(1, light_bytes);
                            if (hv.t1 > hv.t0) {
                                Ln.begin(K_HEAVY);
                                uint64_t *part = (uint64_t *)W(p->off_partial);
                                if (bulk)
                                    launch_gather_tasks_bulk(st, Ls, Lg, hv.t0, hv.t1, g->col_idx, g->nnz, sp.task_e, X,
                                                             R, part, err);
                                else if (group)
                                    launch_gather_tasks_group(st, Ls, Lg, hv.t0, hv.t1, g->col_idx, sp.task_e, X, R,
                                                              part);
                                else if (vec)
                                    launch_gather_tasks_vec(st, Ls, Lg, hv.t0, hv.t1, g->col_idx, sp.task_e, X, R, part);
                                else
                                    launch_gather_tasks(st, Ls, Lg, hv.t0, hv.t1, g->col_idx, sp.task_e, X, R, part,
                                                        gm == 4, gm == 5 ? nullptr : next_counter(), gm == 6 ? 2 : 4,
                                                        column_segments(R, Ls, p->col_chunks), skip_for(s.p));
                                launch_gather_reduce(st, Lg, hv.h0, hv.h1, v0, hv.t0, sp.heavy_v, sp.heavy_tptr, part,
                                                     R, agg);
                                Ln.end(2, heavy_bytes);
                            }
                        };
                        const auto site = std::make_pair((int)ci, (int)si);
                        if (tune) {
                            // every variant computes the same sums; the last one run leaves agg
                            for (int gm : {0, 2, 3, 4, 5, 6, 1}) {  // the default (1) last
                                if ((gm == 0 && !bulk_gather_ok(Ls, R)) || ((gm == 2 || gm == 3) && !vec_gather_ok(Ls, R)))
                                    continue;
                                PlanInstance::Trial tr{(int)ci, (int)si, gm, nullptr, nullptr};
                                cudaEventCreate(&tr.a);
                                cudaEventCreate(&tr.b);
                                cudaEventRecord(tr.a, st);
                                run_gather(gm);
                                cudaEventRecord(tr.b, st);
                                p->trials.push_back(tr);
                            }
                        } else {
                            auto it = p->site_mode.find(site);
                            run_gather(it != p->site_mode.end() ? it->second : c->opt.gather_mode);
                        }
                    }
                    if (s.a == 1) {
                        note_path(si, CC_PATH_GATHER_SELECT, Ls, Lg, Lo);
                        Ln.begin(K_SELECT);
                        // a = 1: the output is the aggregate (Lg == Lo)
                        launch_combine_select(st, Lo, false, v0, nv, B, k, Ch, Chs, Cps, p->d_rm[s.h], col, agg, out);
                        Ln.end(1, (double)nv * B * ((Ch + Cp) * 8.0 * Lo + 1));
                    } else {
                        note_path(si, CC_PATH_GATHER_COMBINE, Ls, Lg, Lo);
                        Ln.begin(K_COMBINE);
                        launch_combine_generic(st, Lo, La, Lg, nv, B, Ch, Chs, cur_stride, Cps, binom(s.h, s.a),
                                               p->d_pairs.at({s.h, s.a}), cur, agg, out, k, col + (uint64_t)v0 * B,
                                               p->d_rm[s.h], p->d_elig.at(s.h), binom(k - 1, s.h - 1));
                        Ln.end(1, (double)nv * B * (Ch * 8.0 * Lo + binom(k, s.a) * 8.0 * La + Cp * 8.0 * Lg));
                    }
                }
                cur = out;
                cur_stride = Chs;
            }
            if (C.label >= 0 && g->labels) {
                // labelled template: the chain's vertex may sit only on vertices with its label
                int64_t Chs_last;
                uint64_t *rows = step_out(C.steps.size() - 1, &Chs_last);
                const int64_t words = (int64_t)B * Chs_last * L;
                Ln.begin(K_SELECT);
                launch_mask_rows(st, nv, words, g->labels + v0, C.label, rows);
                Ln.end(1, (double)nv * (1 + words * 8.0));
            }
            if (C.is_root) {
                Ln.begin(K_REDUCE);
                uint64_t *slot_totals = totals + (size_t)p->chain_slot[ci] * p->n_members * B * p->L_root;
                if (p->n_members > 1)
                    launch_member_reduce(st, p->L_root, v0, v1, B, root_rows, g->member_act, g->n_members,
                                         slot_totals);
                else
                    launch_root_reduce(st, p->L_root, nv, B, root_rows, (uint64_t *)W(p->off_scratch),
                                       reduce_scratch_ctas(), slot_totals);
                int nl = 2;
                if (n_samples > 0) {
                    launch_sample_extract(st, p->L_root, n_samples, d_samples, v0, v1, B, root_rows, d_samples_out);
                    nl++;
                }
                Ln.end(nl, (double)nv * B * 8 * p->L_root);
            }
        }
    }
    CC_CUDA(cudaGetLastError());
    return CC_OK;
}

// Capture one pass (colour .. root reduce) as a CUDA graph; launch counters are
// restored because capturing launches nothing.
static cc_status capture_pass(Ctx *c, PlanInstance *p, char *ws, cudaStream_t st, CachedPlan *cp)
{
    const int64_t l0 = c->launches.load();
    KernelTimer saved = c->timer;
    CC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cc_status rc = launch_pass(c, p, ws, st, nullptr, 0, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    cp->launches_per_pass = c->launches.load() - l0;
    c->launches = l0;
    for (int i = 0; i < CC_KERNEL_KINDS; i++) c->timer.launches[i] = saved.launches[i];
    c->timer.total_launches = saved.total_launches;
    if (rc != CC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&cp->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cp->gexec = nullptr;
        return fail(CC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return CC_OK;
}

// After a tuning pass: per gather site, the variant with the least summed time.
static cc_status finish_tuning(Ctx *c, PlanInstance *p, cudaStream_t st)
{
    CC_CUDA(cudaStreamSynchronize(st));
    std::map<std::pair<int, int>, std::map<int, double>> t;
    for (auto &tr : p->trials) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, tr.a, tr.b) == cudaSuccess) t[{tr.chain, tr.step}][tr.mode] += ms;
        cudaEventDestroy(tr.a);
        cudaEventDestroy(tr.b);
    }
    cudaGetLastError();
    p->trials.clear();
    const bool log = std::getenv("CC_TUNE_LOG") != nullptr;
    for (auto &site : t) {
        int best = c->opt.gather_mode;
        double bt = 1e300;
        for (auto &m : site.second)
            if (m.second < bt) bt = m.second, best = m.first;
        p->site_mode[site.first] = best;
        if (log) {
            std::fprintf(stderr, "cc autotune: chain %d step %d:", site.first.first, site.first.second);
            for (auto &m : site.second) std::fprintf(stderr, " mode %d %.3f ms;", m.first, m.second);
            std::fprintf(stderr, " -> %d\n", best);
        }
    }
    p->tuned = true;
    if (p->tmpl_id >= 0) c->tuned_modes[std::make_tuple(p->graph_id, p->tmpl_id, p->B)] = p->site_mode;
    return CC_OK;
}

cc_status run_passes(Ctx *c, PlanInstance *p, char *ws, const CountJob &job, int pass0, int pass1,
                     cudaStream_t st, ColourParams *host_params, uint64_t *host_totals, uint64_t *host_samples,
                     const int64_t *d_samples, int64_t n_samples, uint64_t *d_samples_out, CachedPlan *graph)
{
    const int B = p->B;
    for (int ps = pass0; ps < pass1; ps++) {
        ColourParams &hp = host_params[ps];
        const uint64_t fs = splitmix64_host(job.seed);
        for (int b = 0; b < B; b++)
            hp.hj[b] = splitmix64_host(fs + (uint64_t)(job.first_iter + (int64_t)ps * B + b));
        CC_CUDA(cudaMemcpyAsync(ws + p->off_params, &hp, sizeof(ColourParams), cudaMemcpyHostToDevice, st));
        const bool tune = c->opt.autotune && !p->tuned;
        if (graph && !graph->gexec && !tune && n_samples == 0) CC_TRY(capture_pass(c, p, ws, st, graph));
        if (graph && graph->gexec && !tune && n_samples == 0) {
            CC_CUDA(cudaGraphLaunch(graph->gexec, st));
            c->launches += graph->launches_per_pass;
            c->timer.total_launches += graph->launches_per_pass;
        } else {
            CC_TRY(launch_pass(c, p, ws, st, d_samples, n_samples, d_samples_out, tune));
            if (tune) CC_TRY(finish_tuning(c, p, st));
        }
        CC_CUDA(cudaMemcpyAsync(host_totals + (size_t)ps * p->totals_words(), ws + p->off_totals,
                                (size_t)p->totals_words() * 8, cudaMemcpyDeviceToHost, st));
        if (n_samples > 0)
            CC_CUDA(cudaMemcpyAsync(host_samples + (size_t)ps * B * n_samples * p->L_root, d_samples_out,
                                    (size_t)B * n_samples * 8 * p->L_root, cudaMemcpyDeviceToHost, st));
        if (c->timer.on) {
            CC_CUDA(cudaStreamSynchronize(st));
            drain_timer(c);
        }
    }
    return CC_OK;
}

cc_status run_pass_with(Ctx *c, PlanInstance *p, char *ws, const ColourParams *host_params, cudaStream_t st,
                        uint64_t *host_totals)
{
    CC_CUDA(cudaMemcpyAsync(ws + p->off_params, host_params, sizeof(ColourParams), cudaMemcpyHostToDevice, st));
    CC_TRY(launch_pass(c, p, ws, st, nullptr, 0, nullptr, false));
    CC_CUDA(cudaMemcpyAsync(host_totals, ws + p->off_totals, (size_t)p->totals_words() * 8, cudaMemcpyDeviceToHost,
                            st));
    if (c->timer.on) {
        CC_CUDA(cudaStreamSynchronize(st));
        drain_timer(c);
    }
    return CC_OK;
}

namespace {

// q = x / d, returns remainder (x has L limbs)
uint64_t divmod_small(const uint64_t *x, int L, uint64_t d, uint64_t *q)
{
    unsigned __int128 r = 0;
    for (int i = L - 1; i >= 0; i--) {
        unsigned __int128 cur = (r << 64) | x[i];
        q[i] = (uint64_t)(cur / d);
        r = cur % d;
    }
    return (uint64_t)r;
}

double to_double(const uint64_t *x, int L)
{
    double d = 0;
    for (int i = L - 1; i >= 0; i--) d = d * 18446744073709551616.0 + (double)x[i];
    return d;
}

}  // namespace

cc_status finish_counts(Ctx *c, PlanInstance *p, Graph *g, const CountJob &job, const uint64_t *totals,
                        const uint64_t *samples, uint64_t *counts, int32_t cap, uint64_t *maps,
                        uint64_t *sample_out, cc_result *res, int tr, int member)
{
    (void)c;
    // totals rows hold L_root limbs; this template's total needs its low L limbs
    const int k = p->tp.k, Lst = p->L_root, L = p->tmpl_L[tr], B = p->B, slot = p->tmpl_slot[tr];
    const int n_iter = job.n_iter;
    const int64_t ns = (int64_t)job.sample_vertices.size();
    cc_result r;
    std::memset(&r, 0, sizeof r);
    r.k = k;
    r.limbs = L;
    r.exact = p->exact ? 1 : 0;
    r.n_iter = n_iter;
    r.aut = p->tmpl_aut[tr];
    r.root = p->tmpl_root[tr];
    r.batch = B;
    r.workspace_bytes = p->ws_bytes;
    if (cap < L) {
        if (res) *res = r;
        return fail(CC_ERR_CAPACITY, "limbs_capacity " + std::to_string(cap) + " < needed " + std::to_string(L));
    }
    std::vector<double> est(n_iter);
    double kk = std::pow((double)k, (double)k), kf = 1;
    for (int i = 2; i <= k; i++) kf *= i;
    std::vector<uint64_t> q(L);
    for (int j = 0; j < n_iter; j++) {
        const int ps = j / B, b = j % B;
        const uint64_t *m = totals + ((((size_t)ps * p->n_slots + slot) * p->n_members + member) * B + b) * Lst;
        if (maps)
            for (int l = 0; l < cap; l++) maps[(size_t)j * cap + l] = l < L ? m[l] : 0;
        if (p->exact) {
            uint64_t rem = divmod_small(m, L, (uint64_t)p->tmpl_aut[tr], q.data());
            if (rem) return fail(CC_ERR_INTERNAL, "labelled map count not divisible by |Aut(T)|");
            for (int l = 0; l < cap; l++) counts[(size_t)j * cap + l] = l < L ? q[l] : 0;
            est[j] = to_double(q.data(), L) * (kk / kf);
        } else {
            for (int l = 0; l < cap; l++) counts[(size_t)j * cap + l] = l < L ? m[l] : 0;
        }
        if (sample_out && ns > 0) {
            for (int64_t s = 0; s < ns; s++) {
                uint64_t *dst = sample_out + ((size_t)j * ns + s) * cap;
                int64_t ov = job.sample_vertices[s];
                int64_t cv = (ov >= 0 && ov < g->n) ? g->h_new_id[ov] : -1;
                for (int l = 0; l < cap; l++) dst[l] = 0;
                if (cv >= 0 && samples) {
                    const uint64_t *src = samples + (((size_t)ps * B + b) * ns + s) * Lst;
                    for (int l = 0; l < L; l++) dst[l] = src[l];
                }
            }
        }
    }
    if (p->exact && n_iter > 0) {
        double s = 0;
        for (double e : est) s += e;
        r.estimate = s / n_iter;
        int t = std::max(1, std::min(job.mom_groups, n_iter));
        int qsz = n_iter / t;
        std::vector<double> means;
        for (int gi = 0; gi < t; gi++) {
            double a = 0;
            for (int i = gi * qsz; i < (gi + 1) * qsz; i++) a += est[i];
            means.push_back(a / qsz);
        }
        std::sort(means.begin(), means.end());
        r.median_of_means = (t % 2) ? means[t / 2] : 0.5 * (means[t / 2 - 1] + means[t / 2]);
    }
    if (res) {
        double dev = res->device_seconds, wall = res->wall_seconds;
        int64_t kl = res->kernel_launches;
        *res = r;
        res->device_seconds = dev;
        res->wall_seconds = wall;
        res->kernel_launches = kl;
    }
    return CC_OK;
}

// special cases with no DP: k = 1 (every vertex, isolated ones included), or no edges
// label: the single vertex's label of a labelled k = 1 template, else -1
static cc_status trivial_counts(Graph *g, const CountJob &job, int k, int64_t aut, uint64_t *counts, int32_t cap,
                                uint64_t *maps, uint64_t *sample_out, cc_result *res, int label = -1)
{
    if (cap < 1) return fail(CC_ERR_CAPACITY, "limbs_capacity < 1");
    if (label >= 0 && g->h_labels.empty())
        return fail(CC_ERR_INVALID_ARG, "labelled template on a graph without vertex labels");
    uint64_t v = (k == 1) ? (uint64_t)g->n : 0;
    if (k == 1 && label >= 0) v = (uint64_t)std::count(g->h_labels.begin(), g->h_labels.end(), (uint8_t)label);
    double kk = std::pow((double)k, (double)k), kf = 1;
    for (int i = 2; i <= k; i++) kf *= i;
    for (int j = 0; j < job.n_iter; j++) {
        for (int l = 0; l < cap; l++) {
            counts[(size_t)j * cap + l] = l == 0 ? v : 0;
            if (maps) maps[(size_t)j * cap + l] = l == 0 ? v : 0;
        }
        for (size_t s = 0; sample_out && s < job.sample_vertices.size(); s++)
            for (int l = 0; l < cap; l++) {
                int64_t ov = job.sample_vertices[s];
                sample_out[((size_t)j * job.sample_vertices.size() + s) * cap + l] =
                    (l == 0 && k == 1 && ov >= 0 && ov < g->n && (label < 0 || g->h_labels[ov] == label)) ? 1 : 0;
            }
    }
    if (res) {
        std::memset(res, 0, sizeof *res);
        res->k = k;
        res->limbs = 1;
        res->exact = 1;
        res->n_iter = job.n_iter;
        res->aut = aut;
        res->estimate = (double)v * kk / kf;
        res->median_of_means = res->estimate;
        res->batch = 1;
    }
    return CC_OK;
}

// Autotuner for the plan's shape: the neighbour-list split threshold
// (Algorithm 4's task size s), the column segments of the gathers and the
// vertex-block size.  A candidate shape is planned, run for one untimed pass
// and then timed over three passes of the count's own first colourings (gather
// variants at their defaults, results discarded); its time is the median.  A
// candidate whose plan or workspace does not fit, or whose pass reports a
// kernel wait that ran out, is skipped; a CUDA error ends the tuning with that
// error.  Coordinate descent: the split threshold first (1024, 4096, 16384),
// then the column segments (the default rule, whole rows, 4 and 16 segments)
// at the best threshold, then the block size (the largest that fits, a half,
// a quarter); options the caller set are not tuned.
static cc_status time_shape(Ctx *c, int64_t gid, int64_t tid, const CountJob &job, int width, cudaStream_t st,
                            const Ctx::TunedShape &shape, double *ms_out)
{
    *ms_out = -1;
    const auto key = std::make_pair(gid, tid);
    auto had = c->tuned_shape.find(key);
    const bool had_shape = had != c->tuned_shape.end();
    const Ctx::TunedShape saved = had_shape ? had->second : Ctx::TunedShape{};
    c->tuned_shape[key] = shape;
    std::unique_ptr<PlanInstance> p;
    cc_status rc = make_plan(c, gid, tid, job.n_iter, width, st, &p);
    if (had_shape)
        c->tuned_shape[key] = saved;
    else
        c->tuned_shape.erase(key);
    if (rc == CC_ERR_BUDGET) return CC_OK;
    if (rc != CC_OK) return rc;
    p->tuned = true;  // no per-site variant trials: time the shape alone
    char *ws = (char *)arena_alloc(c, p->ws_bytes);
    ColourParams *hp = nullptr;
    uint64_t *ht = nullptr;
    std::vector<float> times;
    if (ws && cudaMallocHost(&hp, sizeof(ColourParams)) == cudaSuccess &&
        cudaMallocHost(&ht, (size_t)8 * p->totals_words()) == cudaSuccess) {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        for (int rep = 0; rep < 4 && rc == CC_OK; rep++) {
            cudaMemsetAsync(ws + p->off_err, 0, 256, st);
            cudaEventRecord(a, st);
            rc = run_passes(c, p.get(), ws, job, 0, 1, st, hp, ht, nullptr, nullptr, 0, nullptr, nullptr);
            cudaEventRecord(b, st);
            cudaError_t e = cudaStreamSynchronize(st);
            if (rc == CC_OK && e != cudaSuccess)
                rc = fail(CC_ERR_CUDA, std::string("autotuner pass: ") + cudaGetErrorString(e));
            int kerr = 0;
            if (rc == CC_OK) {
                e = cudaMemcpy(&kerr, ws + p->off_err, sizeof kerr, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) rc = fail(CC_ERR_CUDA, std::string("autotuner: ") + cudaGetErrorString(e));
            }
            if (rc != CC_OK || kerr) {
                times.clear();
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0) times.push_back(ms);  // the first pass warms up
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    cudaStreamSynchronize(st);
    if (hp) cudaFreeHost(hp);
    if (ht) cudaFreeHost(ht);
    if (ws) c->arena.free(ws);
    free_plan(c, p.get());
    if (rc != CC_OK) return rc;
    if (!times.empty()) {
        std::sort(times.begin(), times.end());
        *ms_out = times[times.size() / 2];
    }
    return CC_OK;
}

static cc_status tune_shape(Ctx *c, int64_t gid, int64_t tid, const CountJob &job, int width, cudaStream_t st)
{
    Ctx::TunedShape best;
    double best_ms = -1;
    auto consider = [&](const Ctx::TunedShape &cand) -> cc_status {
        double ms = -1;
        CC_TRY(time_shape(c, gid, tid, job, width, st, cand, &ms));
        if (ms >= 0 && (best_ms < 0 || ms < best_ms)) {
            best_ms = ms;
            best = cand;
        }
        return CC_OK;
    };
    CC_TRY(consider(best));
    if (c->opt.split_threshold <= 0)
        for (int64_t s : {1024, 16384}) {
            Ctx::TunedShape cand = best;
            cand.split = s;
            CC_TRY(consider(cand));
        }
    if (c->opt.col_chunks == 0) {
        const Ctx::TunedShape base = best;
        for (int ch : {1, 4, 16}) {
            Ctx::TunedShape cand = base;
            cand.col_chunks = ch;
            CC_TRY(consider(cand));
        }
    }
    if (c->opt.block_vertices == 0) {
        const Ctx::TunedShape base = best;
        for (int dv : {2, 4}) {
            Ctx::TunedShape cand = base;
            cand.block_div = dv;
            CC_TRY(consider(cand));
        }
    }
    c->tuned_shape[{gid, tid}] = best;
    return CC_OK;
}

cc_status count_sync(Ctx *c, int64_t gid, int64_t tid, const CountJob &job, uint64_t *counts, int32_t cap,
                     uint64_t *maps, uint64_t *sample_out, cc_result *res, double *member_est)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!counts) return fail(CC_ERR_INVALID_ARG, "counts is NULL");
    if (job.n_iter < 0) return fail(CC_ERR_INVALID_ARG, "n_iter < 0");
    auto git = c->graphs.find(gid);
    if (git == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    auto tit = c->templates.find(tid);
    if (tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown template");
    Graph *g = git->second.get();
    Template *t = tit->second.get();
    const int width = job.width_bits >= 0 ? job.width_bits : c->opt.width_bits;
    const bool per_member = member_est != nullptr;
    const int M = per_member ? g->n_members : 1;
    const size_t per = (size_t)job.n_iter * cap;  // counts of one member graph
    if (t->k == 1 || g->n_act == 0 || job.n_iter == 0) {
        CC_TRY(trivial_counts(g, job, t->k, t->aut, counts, cap, maps, sample_out, res,
                              t->labels.empty() ? -1 : t->labels[0]));
        if (per_member && t->k == 1) {
            // k = 1: every vertex of a member graph (with the template's label)
            for (int i = 0; i < M; i++) {
                uint64_t v = 0;
                for (int64_t u = g->h_member_off[i]; u < g->h_member_off[i + 1]; u++)
                    v += t->labels.empty() || g->h_labels[u] == t->labels[0];
                for (int j = 0; j < job.n_iter; j++)
                    for (int l = 0; l < cap; l++) {
                        counts[i * per + (size_t)j * cap + l] = l == 0 ? v : 0;
                        if (maps) maps[i * per + (size_t)j * cap + l] = l == 0 ? v : 0;
                    }
                member_est[i] = (double)v;  // k^k / k! = 1
            }
        } else if (per_member) {
            std::fill(counts, counts + M * per, 0);
            if (maps) std::fill(maps, maps + M * per, 0);
            std::fill(member_est, member_est + M, 0.0);
        }
        return CC_OK;
    }
    cudaStream_t st = c->stream;
    // (autotune is fixed per context, so no plan of (gid, tid) is cached yet)
    if (c->opt.autotune && !c->tuned_shape.count({gid, tid}) &&
        (c->opt.split_threshold <= 0 || c->opt.col_chunks == 0 || c->opt.block_vertices == 0))
        CC_TRY(tune_shape(c, gid, tid, job, width, st));
    const int bcap = std::max(1, std::min({c->opt.batch > 0 ? c->opt.batch : 16, job.n_iter, 64}));
    const auto key = std::make_tuple(gid, tid, bcap, width, per_member);
    CachedPlan *cp = nullptr;
    auto it = c->plan_cache.find(key);
    if (it != c->plan_cache.end()) {
        cp = &it->second;
    } else {
        std::unique_ptr<PlanInstance> np;
        cc_status rc = make_plan(c, gid, tid, job.n_iter, width, st, &np, per_member);
        if (rc == CC_ERR_BUDGET && !c->plan_cache.empty()) {
            evict_plans(c);
            rc = make_plan(c, gid, tid, job.n_iter, width, st, &np, per_member);
        }
        if (rc != CC_OK) return rc;
        char *ws = (char *)c->arena.alloc(np->ws_bytes);
        if (!ws && !c->plan_cache.empty()) {
            evict_plans(c);
            ws = (char *)c->arena.alloc(np->ws_bytes);
        }
        if (!ws) {
            free_plan(c, np.get());
            return fail(CC_ERR_BUDGET, "workspace does not fit the HBM budget");
        }
        CachedPlan &slot = c->plan_cache[key];
        slot.p = std::move(np);
        slot.ws = ws;
        cp = &slot;
    }
    cp->last_use = ++c->use_clock;
    PlanInstance *p = cp->p.get();
    struct Cleanup {
        Ctx *c;
        int64_t *ds = nullptr;
        uint64_t *dso = nullptr;
        void *hp = nullptr, *ht = nullptr, *hs = nullptr;
        ~Cleanup()
        {
            cudaStreamSynchronize(c->stream);
            c->arena.free(ds);
            c->arena.free(dso);
            if (hp) cudaFreeHost(hp);
            if (ht) cudaFreeHost(ht);
            if (hs) cudaFreeHost(hs);
        }
    } cl{c};
    char *ws = cp->ws;
    const int B = p->B;
    const int npass = (job.n_iter + B - 1) / B;
    const int64_t ns = (int64_t)job.sample_vertices.size();
    if (ns > 0) {
        std::vector<int64_t> cv(ns);
        for (int64_t s = 0; s < ns; s++) {
            int64_t ov = job.sample_vertices[s];
            cv[s] = (ov >= 0 && ov < g->n) ? g->h_new_id[ov] : -1;
        }
        cl.ds = (int64_t *)c->arena.alloc(8 * ns);
        cl.dso = (uint64_t *)c->arena.alloc((uint64_t)8 * ns * B * p->L_root);  // (plan in use: no eviction)
        if (!cl.ds || !cl.dso) return fail(CC_ERR_BUDGET, "no room for sampled vertices");
        CC_CUDA(cudaMemcpyAsync(cl.ds, cv.data(), 8 * ns, cudaMemcpyHostToDevice, st));
        CC_CUDA(cudaMemsetAsync(cl.dso, 0, (size_t)8 * ns * B * p->L_root, st));
    }
    CC_CUDA(cudaMallocHost(&cl.hp, sizeof(ColourParams) * npass));
    CC_CUDA(cudaMallocHost(&cl.ht, (size_t)8 * npass * p->totals_words()));
    if (ns > 0) CC_CUDA(cudaMallocHost(&cl.hs, (size_t)8 * npass * B * ns * p->L_root));
    cudaEvent_t e0, e1;
    CC_CUDA(cudaEventCreate(&e0));
    CC_CUDA(cudaEventCreate(&e1));
    int64_t l0 = c->launches.load();
    CC_CUDA(cudaMemsetAsync(ws + p->off_err, 0, 256, st));
    CC_CUDA(cudaEventRecord(e0, st));
    cc_status rc = run_passes(c, p, ws, job, 0, npass, st, (ColourParams *)cl.hp, (uint64_t *)cl.ht,
                              (uint64_t *)cl.hs, cl.ds, ns, cl.dso, (c->opt.use_cuda_graph && !c->timer.on) ? cp : nullptr);
    CC_CUDA(cudaEventRecord(e1, st));
    CC_CUDA(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CC_OK) return rc;
    int kerr = 0;
    CC_CUDA(cudaMemcpy(&kerr, ws + p->off_err, sizeof kerr, cudaMemcpyDeviceToHost));
    if (kerr) return fail(CC_ERR_TIMEOUT, "a gather kernel wait ran out of time (code " + std::to_string(kerr) + ")");
    if (res) {
        res->device_seconds = ms * 1e-3;
        res->kernel_launches = c->launches.load() - l0;
    }
    if (!per_member) {
        rc = finish_counts(c, p, g, job, (const uint64_t *)cl.ht, (const uint64_t *)cl.hs, counts, cap, maps,
                           sample_out, res);
    } else {
        // member graphs one by one; the result's estimate is that of the whole
        // batch (the sum: copies in a disjoint union add up)
        cc_result all{}, one{};
        if (res) all = *res;
        double sum = 0;
        for (int i = 0; i < M && rc == CC_OK; i++) {
            one = all;
            rc = finish_counts(c, p, g, job, (const uint64_t *)cl.ht, i == 0 ? (const uint64_t *)cl.hs : nullptr,
                               counts + i * per, cap, maps ? maps + i * per : nullptr,
                               i == 0 ? sample_out : nullptr, &one, 0, i);
            member_est[i] = one.estimate;
            sum += one.estimate;
        }
        if (res) {
            *res = one;
            res->estimate = res->median_of_means = sum;
        }
    }
    if (res)
        res->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    return rc;
}

cc_status count_multi_sync(Ctx *c, int64_t gid, const std::vector<int64_t> &tids, const CountJob &job,
                           uint64_t *counts, int32_t cap, uint64_t *maps, cc_result *res)
{
    auto t_start = std::chrono::steady_clock::now();
    if (!counts) return fail(CC_ERR_INVALID_ARG, "counts is NULL");
    if (job.n_iter < 0) return fail(CC_ERR_INVALID_ARG, "n_iter < 0");
    if (tids.empty()) return fail(CC_ERR_INVALID_ARG, "no templates");
    if (!job.sample_vertices.empty()) return fail(CC_ERR_INVALID_ARG, "sampled vertices need a single template");
    auto git = c->graphs.find(gid);
    if (git == c->graphs.end()) return fail(CC_ERR_NOT_FOUND, "unknown graph");
    Graph *g = git->second.get();
    std::vector<const Template *> ts;
    for (int64_t tid : tids) {
        auto tit = c->templates.find(tid);
        if (tit == c->templates.end()) return fail(CC_ERR_NOT_FOUND, "unknown template");
        ts.push_back(tit->second.get());
        if (ts.back()->k != ts[0]->k) return fail(CC_ERR_INVALID_ARG, "templates of one count must have the same k");
    }
    const size_t nt = ts.size(), per = (size_t)job.n_iter * cap;
    const int width = job.width_bits >= 0 ? job.width_bits : c->opt.width_bits;
    if (ts[0]->k == 1 || g->n_act == 0 || job.n_iter == 0) {
        for (size_t r = 0; r < nt; r++)
            CC_TRY(trivial_counts(g, job, ts[r]->k, ts[r]->aut, counts + r * per, cap, maps ? maps + r * per : nullptr,
                                  nullptr, res ? res + r : nullptr, ts[r]->labels.empty() ? -1 : ts[r]->labels[0]));
        return CC_OK;
    }
    cudaStream_t st = c->stream;
    std::unique_ptr<PlanInstance> p;
    cc_status rc = make_plan_multi(c, gid, tids, job.n_iter, width, st, &p);
    if (rc == CC_ERR_BUDGET && !c->plan_cache.empty()) {
        evict_plans(c);
        rc = make_plan_multi(c, gid, tids, job.n_iter, width, st, &p);
    }
    if (rc != CC_OK) return rc;
    struct Cleanup {
        Ctx *c;
        PlanInstance *p;
        char *ws = nullptr;
        void *hp = nullptr, *ht = nullptr;
        ~Cleanup()
        {
            cudaStreamSynchronize(c->stream);
            c->arena.free(ws);
            free_plan(c, p);
            if (hp) cudaFreeHost(hp);
            if (ht) cudaFreeHost(ht);
        }
    } cl{c, p.get()};
    cl.ws = (char *)c->arena.alloc(p->ws_bytes);
    if (!cl.ws && !c->plan_cache.empty()) {
        evict_plans(c);
        cl.ws = (char *)c->arena.alloc(p->ws_bytes);
    }
    if (!cl.ws) return fail(CC_ERR_BUDGET, "workspace does not fit the HBM budget");
    const int B = p->B;
    const int npass = (job.n_iter + B - 1) / B;
    CC_CUDA(cudaMallocHost(&cl.hp, sizeof(ColourParams) * npass));
    CC_CUDA(cudaMallocHost(&cl.ht, (size_t)8 * npass * p->totals_words()));
    cudaEvent_t e0, e1;
    CC_CUDA(cudaEventCreate(&e0));
    CC_CUDA(cudaEventCreate(&e1));
    const int64_t l0 = c->launches.load();
    CC_CUDA(cudaMemsetAsync(cl.ws + p->off_err, 0, 256, st));
    CC_CUDA(cudaEventRecord(e0, st));
    rc = run_passes(c, p.get(), cl.ws, job, 0, npass, st, (ColourParams *)cl.hp, (uint64_t *)cl.ht, nullptr, nullptr,
                    0, nullptr, nullptr);
    CC_CUDA(cudaEventRecord(e1, st));
    CC_CUDA(cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CC_OK) return rc;
    int kerr = 0;
    CC_CUDA(cudaMemcpy(&kerr, cl.ws + p->off_err, sizeof kerr, cudaMemcpyDeviceToHost));
    if (kerr) return fail(CC_ERR_TIMEOUT, "a gather kernel wait ran out of time (code " + std::to_string(kerr) + ")");
    for (size_t r = 0; r < nt; r++) {
        cc_result *rr = res ? res + r : nullptr;
        if (rr) {
            std::memset(rr, 0, sizeof *rr);
            rr->device_seconds = ms * 1e-3;  // the shared passes
            rr->kernel_launches = c->launches.load() - l0;
        }
        CC_TRY(finish_counts(c, p.get(), g, job, (const uint64_t *)cl.ht, nullptr, counts + r * per, cap,
                             maps ? maps + r * per : nullptr, nullptr, rr, (int)r));
        if (rr) rr->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    }
    return CC_OK;
}

void *arena_alloc(Ctx *c, uint64_t bytes)
{
    void *p = c->arena.alloc(bytes);
    if (!p && !c->plan_cache.empty()) {
        evict_plans(c);
        p = c->arena.alloc(bytes);
    }
    return p;
}

void evict_plans(Ctx *c, int64_t gid, int64_t tid)
{
    cudaStreamSynchronize(c->stream);
    for (auto it = c->tuned_modes.begin(); it != c->tuned_modes.end();) {
        if ((gid >= 0 && std::get<0>(it->first) == gid) || (tid >= 0 && std::get<1>(it->first) == tid))
            it = c->tuned_modes.erase(it);
        else
            ++it;
    }
    for (auto it = c->plan_cache.begin(); it != c->plan_cache.end();) {
        const bool hit = (gid < 0 && tid < 0) || std::get<0>(it->first) == gid || std::get<1>(it->first) == tid;
        if (!hit) {
            ++it;
            continue;
        }
        if (it->second.gexec) cudaGraphExecDestroy(it->second.gexec);
        for (auto &tr : it->second.p->trials) {
            cudaEventDestroy(tr.a);
            cudaEventDestroy(tr.b);
        }
        c->arena.free(it->second.ws);
        free_plan(c, it->second.p.get());
        it = c->plan_cache.erase(it);
    }
}

}  // namespace cc
