// runtime.h -- context, graphs, templates, plan instances and the executor.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"
#include "kernels.cuh"
#include "plan.h"

namespace cc {

// thread-local error message; returns the status for `return fail(...)`
cc_status fail(cc_status s, const std::string &msg);

#define CC_CUDA(call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return ::cc::fail(CC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

#define CC_TRY(expr)                      \
    do {                                  \
        cc_status s_ = (expr);            \
        if (s_ != CC_OK) return s_;       \
    } while (0)

// Best-fit sub-allocator over one device allocation (256-byte aligned blocks).
class Arena {
public:
    void init(char *base, uint64_t bytes);
    // returns nullptr when no free block is large enough
    void *alloc(uint64_t bytes);
    void free(void *p);
    uint64_t free_bytes() const { return free_total_; }
    uint64_t largest_free() const;
    uint64_t capacity() const { return cap_; }
    char *base() const { return base_; }

private:
    char *base_ = nullptr;
    uint64_t cap_ = 0, free_total_ = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> size
    std::map<uint64_t, uint64_t> used_;  // offset -> size
};

struct Graph {
    int64_t n = 0, n_act = 0, nnz = 0;
    int64_t max_degree = 0;
    // device (arena)
    int64_t *row_ptr = nullptr;   // [n_act + 1]
    int32_t *col_idx = nullptr;   // [nnz], compact ids
    int64_t *orig = nullptr;      // [n_act] id of each compact vertex that its colour is drawn from:
                                  // its input id, or its id within its member graph (graph batches)
    // host copies used for planning
    std::vector<int64_t> h_row_ptr;
    std::vector<int32_t> h_new_id;  // original id -> compact id or -1 (isolated)
    // graph batches: member graph i holds input ids [h_member_off[i],
    // h_member_off[i + 1]) and compact ids [h_member_act[i], h_member_act[i + 1])
    // (compact ids are ordered by member first); one member otherwise
    int32_t n_members = 1;
    std::vector<int64_t> h_member_off, h_member_act;
    int64_t *member_act = nullptr;  // device copy of h_member_act [n_members + 1]
    // vertex labels for labelled templates, or none: host copy in the original
    // numbering [n], device copy in the compact numbering [n_act]
    std::vector<uint8_t> h_labels;
    uint8_t *labels = nullptr;
    // homomorphism bounds cache, keyed by a chain's rooted canonical form and
    // the forms of the children it attaches in step order: log2 of max_v and
    // sum_v of the final bound, and per step log2 max_v of the bound after the
    // step and of the step's factor sum_{u in N(v)} H_child(u)
    struct HomBound {
        double l2max = -1, l2sum = -1;
        std::vector<std::pair<double, double>> steps;
    };
    std::map<std::string, HomBound> hom_cache;
    // heavy-vertex task lists per split threshold
    struct Split {
        int64_t s = 0;
        int32_t *heavy_v = nullptr;     // [H]
        int64_t *heavy_tptr = nullptr;  // [H + 1]
        int64_t *task_e = nullptr;      // [2 T]
        std::vector<int32_t> h_heavy_v;
        std::vector<int64_t> h_heavy_tptr;
        int64_t H = 0, T = 0;
    };
    std::map<int64_t, Split> splits;
    int in_use = 0;  // requests referencing this graph
};

struct Template {
    int k = 0, root_req = -1;
    std::vector<int32_t> edges;
    std::vector<uint8_t> labels;  // vertex labels, or empty (unlabelled)
    int64_t aut = 1;              // label-preserving automorphisms when labelled
    std::string canon;            // tree_canonical_form: equal for isomorphic templates
};

// A template planned against a graph with a batch size and width policy.
struct PlanInstance {
    TemplatePlan tp;
    int64_t graph_id = 0, tmpl_id = 0;
    int B = 1;
    int width_bits = 0;     // 0 exact
    bool exact = true;
    int L_root = 1;
    std::vector<int> chain_L;
    // per chain and step: limbs of the step's output rows and of its aggregate
    // (the last step's output is the chain's table, chain_L limbs)
    std::vector<std::vector<int>> step_L, agg_L;
    int Lmax = 1;
    int64_t V = 0;          // vertices per block
    std::vector<std::pair<int64_t, int64_t>> blocks;
    // heavy vertices [h0, h1) of the heavy list, their tasks [t0, t1), and the
    // edges of their neighbour lists
    struct BlockHeavy { int64_t h0, h1, t0, t1, edges; };
    std::vector<BlockHeavy> heavy;
    int64_t split = 1024;
    int col_chunks = 0;     // column segments in use (cc_options.col_chunks meaning)
    bool shape_tuned = false;
    int64_t max_tasks = 0;
    // device constants (arena): rm tables per h, pair tables per (h, a)
    void *consts = nullptr;
    std::vector<uint16_t *> d_rm;               // [h]
    std::vector<uint16_t *> d_ad;               // [p] (fused gather + select steps)
    std::map<std::pair<int, int>, uint32_t *> d_pairs;
    std::map<int, uint16_t *> d_elig;           // [h]: per colour, the ranks of the h-sets holding it
    std::vector<uint16_t *> d_smask;            // [h]: colour mask of each column (AbsentSkip), 0 padding
    // workspace layout (offsets from ws base)
    uint64_t ws_bytes = 0;
    // workspace of the same plan with every table kept for the whole pass, with
    // one vertex block, and with both (analytic; nothing is allocated)
    uint64_t ws_no_reuse = 0, ws_no_blocks = 0, ws_naive = 0;
    uint64_t off_col = 0, off_hist = 0, off_act[2] = {0, 0}, off_agg = 0, off_partial = 0, off_root = 0,
             off_scratch = 0, off_totals = 0, off_params = 0, off_err = 0, off_ctr = 0;
    uint64_t off_ncol = ~0ull;        // neighbour colours of the pass (AbsentSkip), ~0: whole rows
    bool absent_skip = false;         // the plan may skip absent entries (batch 1 decides)
    std::vector<uint64_t> off_table;  // per chain (materialised), ~0 for root
    // analytic figures
    double updates = 0, gather_bytes = 0, alg_bytes = 0, pairs = 0, limb_products = 0;
    // autotuner: gather kernel variant per gather site (chain, step), chosen by
    // timing every applicable variant on the first pass
    std::map<std::pair<int, int>, int> site_mode;
    bool tuned = false;
    struct Trial { int chain, step, mode; cudaEvent_t a, b; };
    std::vector<Trial> trials;
    // Root chains and templates.  Every distinct root chain sums into its own
    // totals slot (n_slots x B x L_root values per pass).  Template r of the
    // plan (one, or several sharing their colourings) reads slot tmpl_slot[r],
    // keeps its low tmpl_L[r] limbs (exact: its total is below 2^(64 tmpl_L[r]))
    // and divides by tmpl_aut[r].
    // colour histograms: one per distinct label of leaf children (-1: all
    // neighbours, unlabelled templates), n_act x B x k counts each
    std::vector<int> hist_labels;
    int n_slots = 1;
    // graph batches: every slot holds n_members totals (one per member graph):
    // totals are [n_slots][n_members][B][L_root] per pass
    int n_members = 1;
    int64_t totals_words() const { return (int64_t)n_slots * n_members * B * L_root; }
    std::vector<int> chain_slot;     // per chain: totals slot, -1 for non-root chains
    std::vector<int> tmpl_slot, tmpl_L, tmpl_root;
    std::vector<int64_t> tmpl_aut;
    // how the last pass ran each (chain, step) for the light vertices of the
    // first vertex block: a CC_PATH_* code and the kernel's limb arguments
    struct StepPath { int path = 0, l0 = 0, l1 = 0, l2 = 0; };
    std::vector<std::vector<StepPath>> step_path;
    // several templates: chains and gathered updates per colouring had each
    // been planned alone
    int sep_chains = 0;
    double sep_updates = 0;
};

enum KernelKind { K_COLOUR = 0, K_HIST, K_GATHER, K_COMBINE, K_REDUCE, K_FUSED, K_SELECT, K_CHIST, K_HEAVY, K_KINDS };

struct KernelTimer {
    bool on = false;
    int64_t launches[CC_KERNEL_KINDS] = {0};
    double seconds[CC_KERNEL_KINDS] = {0};
    double bytes[CC_KERNEL_KINDS] = {0};
    int64_t total_launches = 0;
    // kernel instantiations launched under each kind (note_launch names):
    // launches, and the time and algorithmic bytes of the timed brackets that
    // launched that instantiation alone
    struct Inst { int64_t launches = 0, timed_launches = 0; double seconds = 0, bytes = 0; };
    std::map<std::string, Inst> instances[CC_KERNEL_KINDS];
    struct Pending { cudaEvent_t a, b; int kind; double bytes; std::string only; int64_t n; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
};

struct Request;

// A plan kept between cc_count calls with its workspace and, when enabled, the
// per-pass schedule captured as a CUDA graph (pointers into the workspace are
// fixed, so the graph can be replayed with new colouring parameters).
struct CachedPlan {
    std::unique_ptr<PlanInstance> p;
    char *ws = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t launches_per_pass = 0;
    uint64_t last_use = 0;
};

struct Ctx {
    cc_options opt;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char *arena_base = nullptr;
    bool own_arena = false;
    Arena arena;
    std::recursive_mutex mu;
    int64_t next_id = 1;
    std::map<int64_t, std::unique_ptr<Graph>> graphs;
    std::map<int64_t, std::unique_ptr<Template>> templates;
    KernelTimer timer;
    std::atomic<int64_t> launches{0};
    // plans kept between calls: (graph, template, batch cap, width) -> plan
    // (graph, template, batch cap, width bits, per-member totals)
    std::map<std::tuple<int64_t, int64_t, int, int, bool>, CachedPlan> plan_cache;
    uint64_t use_clock = 0;
    // autotuned gather variants per (graph, template, batch), shared by later plans
    std::map<std::tuple<int64_t, int64_t, int>, std::map<std::pair<int, int>, int>> tuned_modes;
    // autotuned plan shape per (graph, template): neighbour-list split
    // threshold, column segments (0: the default rule) and the divisor of the
    // largest vertex block that fits (1: the largest)
    struct TunedShape { int64_t split = 4096; int col_chunks = 0; int block_div = 1; };
    std::map<std::pair<int64_t, int64_t>, TunedShape> tuned_shape;
    // serving
    std::unique_ptr<struct Server> server;
    uint64_t l2_window_bytes = 0;  // cc_options.l2_persist_mb as granted (0: no access window)
    Ctx();
    ~Ctx();  // defined where Server is complete
};

// executor entry points
// member_off: NULL (one graph) or n_members + 1 increasing input-id offsets
// starting at 0 and ending at n (a batch of member graphs, no edge between two)
cc_status graph_load(Ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                     cc_graph_id *out, int32_t n_members = 1, const int64_t *member_off = nullptr);
cc_status graph_free(Ctx *c, Graph *g);
cc_status ensure_split(Ctx *c, Graph *g, int64_t s, cudaStream_t st);

struct CountJob {
    uint64_t seed = 0;
    int64_t first_iter = 0;
    int32_t n_iter = 0;
    int32_t width_bits = -1;
    int32_t mom_groups = 1;
    std::vector<int64_t> sample_vertices;  // original ids
};

// plan (with workspace sizing) for a count with n_iter colourings
// per_member: one total per member graph of a graph batch (else one for the
// whole graph)
cc_status make_plan(Ctx *c, int64_t gid, int64_t tid, int n_iter, int width_bits, cudaStream_t st,
                    std::unique_ptr<PlanInstance> *out, bool per_member = false);
// one plan for several templates with the same k over the same colourings:
// rooted subtrees with equal canonical forms share one table
cc_status make_plan_multi(Ctx *c, int64_t gid, const std::vector<int64_t> &tids, int n_iter, int width_bits,
                          cudaStream_t st, std::unique_ptr<PlanInstance> *out);
// counts of several templates (counts, maps: [template][colouring][cap]; res: [template])
cc_status count_multi_sync(Ctx *c, int64_t gid, const std::vector<int64_t> &tids, const CountJob &job,
                           uint64_t *counts, int32_t cap, uint64_t *maps, cc_result *res);
void free_plan(Ctx *c, PlanInstance *p);

// Runs passes [pass0, pass1) of a job on stream st using workspace ws.
// Per pass: host params -> device, colour, hist, chains, reduce; totals/samples
// copied to host_totals / host_samples (pinned) at pass offsets.
cc_status run_passes(Ctx *c, PlanInstance *p, char *ws, const CountJob &job, int pass0, int pass1,
                     cudaStream_t st, ColourParams *host_params, uint64_t *host_totals, uint64_t *host_samples,
                     const int64_t *d_samples, int64_t n_samples, uint64_t *d_samples_out,
                     CachedPlan *graph = nullptr);

// One pass with the given colouring parameters (host_params[0].hj[b] for the
// plan's B colourings; pinned memory), queued on st: totals of the pass go to
// host_totals (pinned, p->totals_words() words).  The serving loop fills
// the parameters with colourings of several requests.
cc_status run_pass_with(Ctx *c, PlanInstance *p, char *ws, const ColourParams *host_params, cudaStream_t st,
                        uint64_t *host_totals);

// Host post-processing for template tr of the plan: copies, estimate, median
// of means, writes caller buffers.
cc_status finish_counts(Ctx *c, PlanInstance *p, Graph *g, const CountJob &job, const uint64_t *totals,
                        const uint64_t *samples, uint64_t *counts, int32_t cap, uint64_t *maps,
                        uint64_t *sample_out, cc_result *res, int tr = 0, int member = 0);

// member_est: NULL, or a graph batch counted per member graph: counts and maps
// are [n_members][n_iter][cap], member_est[i] the estimate of member i
cc_status count_sync(Ctx *c, int64_t gid, int64_t tid, const CountJob &job, uint64_t *counts, int32_t cap,
                     uint64_t *maps, uint64_t *sample_out, cc_result *res, double *member_est = nullptr);

// drop cached plans (all, or those of one graph / template); frees their workspace
void evict_plans(Ctx *c, int64_t gid = -1, int64_t tid = -1);
// arena allocation that drops cached plans and retries once when the arena is full
void *arena_alloc(Ctx *c, uint64_t bytes);

// serving (serve.cpp)
cc_status serve_submit(Ctx *c, const cc_request *r, cc_req_id *out);
cc_status serve_poll(Ctx *c, cc_req_id id, cc_result *res, uint64_t *counts, int32_t cap, bool wait,
                     int64_t timeout_ns);
cc_status serve_cancel(Ctx *c, cc_req_id id);
cc_status serve_stats(Ctx *c, cc_serve_stats *out);
void serve_shutdown(Ctx *c);

uint64_t splitmix64_host(uint64_t state);

cc_status table_gather(Ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X,
                       uint64_t *agg, int64_t values, int32_t limbs, int32_t split);

}  // namespace cc
