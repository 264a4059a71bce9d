// plan.h -- host-side planning of the colour-coding DP for one tree template.
//
// Section 2.1 of arXiv 1804.09764: the template T is rooted at rho(T) and split
// recursively by cutting one root edge; the part that keeps the root is the
// active child T', the part hanging from the cut neighbour is the passive child
// T''.  Here every template vertex x owns a chain: starting from the single
// vertex x, its children are attached one at a time; each attachment is one
// application of Eq. 1 (a gather over N(v) of the child's table, then a
// disjoint colour-set combine).  The complete subtree table of x is the last
// link of its chain.  Rooted-isomorphic subtrees (same AHU canonical form)
// share one table.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

namespace cc {

constexpr int kMaxK = 16;

int64_t binom(int n, int r);

struct Step {
    int child = -1;        // template vertex attached by this step
    int src_chain = -1;    // chain index holding the child's table; -1: leaf (colour histogram)
    int h = 0, a = 0, p = 0;  // |T_i|, |T_i'|, |T_i''|
    bool reuse_agg = false;   // same source as the previous step: aggregate already on hand
    int leaf_label = -1;      // leaf child: its vertex label (-1: unlabelled template)
};

struct ChainPlan {
    int vertex = -1;       // representative template vertex
    int size = 1;          // vertices in its subtree
    bool is_root = false;
    std::string canon;     // AHU canonical form of the rooted subtree
    std::vector<Step> steps;
    int last_consumer = -1;  // last chain index that gathers this table
    int limbs = 1;           // 64-bit limbs of this chain's values
    int max_cols = 1;        // widest intermediate row (colour-set columns)
    int label = -1;          // vertex label of the chain's template vertex (-1: unlabelled)
};

struct TemplatePlan {
    int k = 0, root = 0;
    int64_t aut = 1;
    std::vector<std::pair<int, int>> edges;
    std::vector<ChainPlan> chains;  // post-order, root chain last
    int64_t table4_memory = 0, table4_computation = 0;
    double pairs_per_vertex = 0;    // sum over steps of the combine work per vertex
};

// Validates and plans.  root = -1 lets the planner choose (cost model with the
// given average degree).  order_mode: 0 = children largest subtree first
// (Table 4's convention), 1 = planner's order (least combine work).
// labels: optional vertex labels (canonical forms and |Aut| then respect them).
// Returns 0, or a negative cc_status with *err set.
int build_template_plan(int k, const int32_t *edges, int root, int order_mode, double avg_degree,
                        TemplatePlan *out, std::string *err, const uint8_t *labels = nullptr);

// |Aut(T)| from AHU canonical forms at the centre of the tree (label-preserving
// automorphisms when labels are given).
int64_t tree_automorphisms(int k, const std::vector<std::vector<int>> &adj, const uint8_t *labels = nullptr);

// Canonical form of an unrooted tree (label-respecting when labels are given):
// the least AHU form of the tree rooted at one of its centres.  Two trees have
// the same form exactly when they are isomorphic (by a label-preserving map),
// and isomorphic templates have the same copy counts in every graph.
std::string tree_canonical_form(int k, const std::vector<std::vector<int>> &adj, const uint8_t *labels = nullptr);

// Colex ranking of k-colour sets (combinatorial number system):
// rank(S) = sum_i C(c_i, i+1) over the members c_0 < c_1 < ... of S.
struct SetTables {
    int k = 0;
    // rm[h] : C(k,h) x k entries, rank of S \ {c} in the (h-1)-sets, or 0xFFFF if c not in S
    std::vector<std::vector<uint16_t>> rm;
    // ad[p] : C(k,p) x k entries, rank of T u {c} in the (p+1)-sets, or 0xFFFF if c in T
    std::vector<std::vector<uint16_t>> ad;
    // members of each set by rank, per size (bitmask)
    std::vector<std::vector<uint32_t>> mask_of_rank;
    void build(int k_);
    // pair table for (h, a): for i in [0, C(h,a)) and S in [0, C(k,h)):
    // entry[i * C(k,h) + S] = rank_a(S_a) | rank_p(S \ S_a) << 16, S_a = i-th a-subset of S
    std::vector<uint32_t> pairs(int h, int a) const;
};

uint32_t colex_rank(uint32_t mask);

}  // namespace cc
