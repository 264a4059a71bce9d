// plan.cpp -- template partition, rooted-isomorphism dedupe, automorphisms,
// colex ranking tables.  Host code only.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>

#include "../../include/cc.h"

namespace cc {

int64_t binom(int n, int r)
{
    if (r < 0 || r > n) return 0;
    int64_t v = 1;
    for (int i = 1; i <= r; i++) v = v * (n - r + i) / i;
    return v;
}

uint32_t colex_rank(uint32_t mask)
{
    uint32_t r = 0;
    int i = 0;
    for (int c = 0; mask; c++, mask >>= 1)
        if (mask & 1) r += (uint32_t)binom(c, ++i);
    return r;
}

void SetTables::build(int k_)
{
    k = k_;
    mask_of_rank.assign(k + 1, {});
    for (int h = 0; h <= k; h++) mask_of_rank[h].resize((size_t)binom(k, h));
    for (uint32_t m = 0; m < (1u << k); m++) {
        int h = __builtin_popcount(m);
        mask_of_rank[h][colex_rank(m)] = m;
    }
    ad.assign(k + 1, {});
    for (int q = 0; q < k; q++) {
        auto &t = ad[q];
        t.assign((size_t)binom(k, q) * k, 0xFFFF);
        for (size_t s = 0; s < mask_of_rank[q].size(); s++) {
            uint32_t m = mask_of_rank[q][s];
            for (int c = 0; c < k; c++)
                if (!(m >> c & 1)) t[s * k + c] = (uint16_t)colex_rank(m | (1u << c));
        }
    }
    rm.assign(k + 1, {});
    for (int h = 1; h <= k; h++) {
        auto &t = rm[h];
        t.assign((size_t)binom(k, h) * k, 0xFFFF);
        for (size_t s = 0; s < mask_of_rank[h].size(); s++) {
            uint32_t m = mask_of_rank[h][s];
            for (int c = 0; c < k; c++)
                if (m >> c & 1) t[s * k + c] = (uint16_t)colex_rank(m & ~(1u << c));
        }
    }
}

std::vector<uint32_t> SetTables::pairs(int h, int a) const
{
    const int64_t nh = binom(k, h), na = binom(h, a);
    std::vector<uint32_t> out((size_t)(nh * na));
    for (int64_t s = 0; s < nh; s++) {
        uint32_t m = mask_of_rank[h][s];
        int pos[kMaxK], np = 0;
        for (int c = 0; c < k; c++)
            if (m >> c & 1) pos[np++] = c;
        // a-subsets of the h members, in colex order of their local patterns
        int64_t i = 0;
        for (uint32_t t = 0; t < (1u << h); t++) {
            if (__builtin_popcount(t) != a) continue;
            uint32_t sa = 0;
            for (int b = 0; b < h; b++)
                if (t >> b & 1) sa |= 1u << pos[b];
            uint32_t sp = m & ~sa;
            out[(size_t)(i * nh + s)] = colex_rank(sa) | (colex_rank(sp) << 16);
            i++;
        }
    }
    return out;
}

namespace {

struct Rooted {
    int k;
    const uint8_t *label = nullptr;  // vertex labels (part of the canonical forms) or none
    std::vector<std::vector<int>> adj, children;
    std::vector<int> parent, size;
    std::vector<std::string> canon;
    std::vector<int> post;  // post-order
};

void root_at(Rooted &R, int root)
{
    R.children.assign(R.k, {});
    R.parent.assign(R.k, -1);
    R.size.assign(R.k, 1);
    R.canon.assign(R.k, "");
    R.post.clear();
    std::function<void(int, int)> dfs = [&](int x, int p) {
        R.parent[x] = p;
        for (int y : R.adj[x])
            if (y != p) {
                R.children[x].push_back(y);
                dfs(y, x);
                R.size[x] += R.size[y];
            }
        std::vector<std::string> cs;
        for (int y : R.children[x]) cs.push_back(R.canon[y]);
        std::sort(cs.begin(), cs.end());
        std::string s = "(";
        if (R.label) s += std::to_string((int)R.label[x]) + ":";
        for (auto &c : cs) s += c;
        R.canon[x] = s + ")";
        R.post.push_back(x);
    };
    dfs(root, -1);
}

// rooted automorphisms: product over vertices of the factorials of the
// multiplicities of identical child subtrees
int64_t rooted_aut(const Rooted &R, int x)
{
    int64_t a = 1;
    std::map<std::string, int> mult;
    for (int y : R.children[x]) {
        a *= rooted_aut(R, y);
        mult[R.canon[y]]++;
    }
    for (auto &kv : mult)
        for (int i = 2; i <= kv.second; i++) a *= i;
    return a;
}

int64_t step_cost(int k, int h, int a) { return binom(k, h) * binom(h, a); }

}  // namespace

// the one or two centres of a tree (the vertices left after stripping leaves
// layer by layer)
static std::vector<int> tree_centres(int k, const std::vector<std::vector<int>> &adj)
{
    std::vector<int> deg(k);
    for (int i = 0; i < k; i++) deg[i] = (int)adj[i].size();
    std::vector<int> layer, removed(k, 0);
    for (int i = 0; i < k; i++)
        if (deg[i] <= 1) layer.push_back(i);
    int left = k;
    while (left > 2) {
        std::vector<int> next;
        for (int x : layer) {
            removed[x] = 1;
            left--;
            for (int y : adj[x])
                if (!removed[y] && --deg[y] == 1) next.push_back(y);
        }
        layer = next;
    }
    std::vector<int> centres;
    for (int i = 0; i < k; i++)
        if (!removed[i]) centres.push_back(i);
    return centres;
}

std::string tree_canonical_form(int k, const std::vector<std::vector<int>> &adj, const uint8_t *labels)
{
    if (k == 1) return labels ? "(" + std::to_string((int)labels[0]) + ":)" : "()";
    std::string best;
    for (int c : tree_centres(k, adj)) {
        Rooted R;
        R.k = k;
        R.label = labels;
        R.adj = adj;
        root_at(R, c);
        if (best.empty() || R.canon[c] < best) best = R.canon[c];
    }
    return std::to_string(k) + best;
}

int64_t tree_automorphisms(int k, const std::vector<std::vector<int>> &adj, const uint8_t *labels)
{
    if (k <= 2) return k == 2 ? (labels && labels[0] != labels[1] ? 1 : 2) : 1;
    const std::vector<int> centres = tree_centres(k, adj);
    Rooted R;
    R.k = k;
    R.label = labels;
    R.adj = adj;
    if (centres.size() == 1) {
        root_at(R, centres[0]);
        return rooted_aut(R, centres[0]);
    }
    // bicentral: cut the central edge, compare the halves
    int c1 = centres[0], c2 = centres[1];
    auto cut = adj;
    cut[c1].erase(std::find(cut[c1].begin(), cut[c1].end(), c2));
    cut[c2].erase(std::find(cut[c2].begin(), cut[c2].end(), c1));
    R.adj = cut;
    root_at(R, c1);
    int64_t a1 = rooted_aut(R, c1);
    std::string s1 = R.canon[c1];
    Rooted R2;
    R2.k = k;
    R2.label = labels;
    R2.adj = cut;
    root_at(R2, c2);
    int64_t a2 = rooted_aut(R2, c2);
    return a1 * a2 * (s1 == R2.canon[c2] ? 2 : 1);
}

int build_template_plan(int k, const int32_t *edges, int root, int order_mode, double avg_degree,
                        TemplatePlan *out, std::string *err, const uint8_t *labels)
{
    if (k < 1 || k > kMaxK) {
        *err = "k must be in 1..16";
        return CC_ERR_K_RANGE;
    }
    if (k > 1 && !edges) {
        *err = "edges is NULL";
        return CC_ERR_INVALID_ARG;
    }
    Rooted R;
    R.k = k;
    R.label = labels;
    R.adj.assign(k, {});
    std::vector<std::pair<int, int>> E;
    for (int e = 0; e < k - 1; e++) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b ||
            std::find(R.adj[a].begin(), R.adj[a].end(), b) != R.adj[a].end()) {
            *err = "template edge list is not a simple graph on 0..k-1";
            return CC_ERR_NOT_TREE;
        }
        R.adj[a].push_back(b);
        R.adj[b].push_back(a);
        E.push_back({a, b});
    }
    {   // connectivity
        std::vector<int> seen(k, 0), st{0};
        seen[0] = 1;
        int cnt = 0;
        while (!st.empty()) {
            int x = st.back();
            st.pop_back();
            cnt++;
            for (int y : R.adj[x])
                if (!seen[y]) seen[y] = 1, st.push_back(y);
        }
        if (cnt != k) {
            *err = "template is not connected";
            return CC_ERR_NOT_TREE;
        }
    }
    for (auto &v : R.adj) std::sort(v.begin(), v.end());
    if (root < -1 || root >= k) {
        *err = "root out of range";
        return CC_ERR_INVALID_ARG;
    }

    // plan for one root; returns modelled cost
    auto plan_root = [&](int r, TemplatePlan &P) -> double {
        root_at(R, r);
        P = TemplatePlan();
        P.k = k;
        P.root = r;
        P.edges = E;
        // order children of every vertex
        std::vector<std::vector<int>> order(k);
        for (int x = 0; x < k; x++) {
            auto ch = R.children[x];
            auto key_less = [&](int u, int w) {
                if (R.size[u] != R.size[w]) return R.size[u] > R.size[w];  // largest first
                return R.canon[u] < R.canon[w];
            };
            std::sort(ch.begin(), ch.end(), key_less);
            if (order_mode == 1 && ch.size() > 1 && ch.size() <= 7) {
                // least combine work; identical subtrees adjacent wins ties
                std::vector<int> best = ch, cur = ch;
                auto cost_of = [&](const std::vector<int> &o) {
                    int64_t c = 0;
                    int a = 1;
                    for (size_t i = 0; i < o.size(); i++) {
                        int h = a + R.size[o[i]];
                        c = c * 1 + step_cost(k, h, a);
                        if (i && R.canon[o[i]] == R.canon[o[i - 1]]) c -= 1;  // aggregate reuse
                        a = h;
                    }
                    return c;
                };
                int64_t bc = cost_of(best);
                // permutations of the sorted sequence over (size, canon) keys
                std::vector<int> idx(cur.size());
                for (size_t i = 0; i < idx.size(); i++) idx[i] = (int)i;
                auto cmp = [&](int i, int j) { return key_less(ch[i], ch[j]); };
                std::sort(idx.begin(), idx.end(), cmp);
                do {
                    for (size_t i = 0; i < idx.size(); i++) cur[i] = ch[idx[i]];
                    int64_t c = cost_of(cur);
                    if (c < bc) bc = c, best = cur;
                } while (std::next_permutation(idx.begin(), idx.end(), [&](int i, int j) {
                    // compare by key so equal subtrees are not permuted among themselves
                    if (R.size[ch[i]] != R.size[ch[j]]) return R.size[ch[i]] > R.size[ch[j]];
                    return R.canon[ch[i]] < R.canon[ch[j]];
                }));
                ch = best;
            }
            order[x] = ch;
        }
        // chains: one per distinct canonical form of non-leaf non-root subtrees, plus root
        std::map<std::string, int> chain_of;
        std::vector<int> chain_for_vertex(k, -1);
        for (int x : R.post) {
            bool leaf = R.children[x].empty();
            if (x != r && leaf) continue;
            if (x != r) {
                auto it = chain_of.find(R.canon[x]);
                if (it != chain_of.end()) {
                    chain_for_vertex[x] = it->second;
                    continue;
                }
            }
            ChainPlan C;
            C.vertex = x;
            C.size = R.size[x];
            C.is_root = (x == r);
            C.canon = R.canon[x];
            C.label = labels ? labels[x] : -1;
            int a = 1;
            C.max_cols = (int)binom(k, 1);
            int prev_src = -2;
            for (int y : order[x]) {
                Step s;
                s.child = y;
                s.src_chain = R.children[y].empty() ? -1 : chain_for_vertex[y];
                s.a = a;
                s.p = R.size[y];
                s.h = a + s.p;
                s.reuse_agg = (s.src_chain == prev_src);
                if (s.src_chain < 0 && labels) s.leaf_label = labels[y];
                prev_src = s.src_chain;
                C.max_cols = std::max<int>(C.max_cols, (int)binom(k, s.h));
                C.steps.push_back(s);
                a = s.h;
            }
            int id = (int)P.chains.size();
            P.chains.push_back(C);
            chain_for_vertex[x] = id;
            if (x != r) chain_of[R.canon[x]] = id;
        }
        // last consumers
        for (size_t c = 0; c < P.chains.size(); c++)
            for (auto &s : P.chains[c].steps)
                if (s.src_chain >= 0) P.chains[s.src_chain].last_consumer = (int)c;
        // Table 4 numbers over the full partition (every vertex's chain, no dedupe)
        double pairs = 0, gather = 0;
        for (int x = 0; x < k; x++) {
            int a = 1;
            for (int y : order[x]) {
                int h = a + R.size[y];
                if (h > 1 && h < k) {
                    P.table4_memory += binom(k, h);
                    P.table4_computation += binom(k, h) * binom(h, a);
                }
                a = h;
            }
        }
        for (auto &C : P.chains)
            for (auto &s : C.steps) {
                pairs += (double)(s.a == 1 ? binom(k, s.h) : binom(k, s.h) * binom(s.h, s.a));
                if (s.src_chain >= 0 && !s.reuse_agg) gather += (double)binom(k, s.p);
            }
        P.pairs_per_vertex = pairs;
        return avg_degree * gather * 8.0 + 6.0 * pairs;
    };

    TemplatePlan best;
    if (root >= 0) {
        plan_root(root, best);
    } else {
        double bc = 1e300;
        for (int r = 0; r < k; r++) {
            TemplatePlan P;
            double c = plan_root(r, P);
            if (c < bc) bc = c, best = P;
        }
    }
    best.aut = tree_automorphisms(k, R.adj, labels);
    *out = best;
    return 0;
}

}  // namespace cc
