/*
 * cc_oracle.c -- plain, slow, single-threaded CPU oracle for the colour-coding
 * dynamic program that counts non-induced tree templates (arXiv 1804.09764,
 * Section 2.1, Eq. 1 and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code with the
 * CUDA path: its own colour-set indexing (a lookup filled by enumerating
 * bitmasks), its own colouring generator, its own 256-bit integers, its own
 * automorphism counter.
 *
 * What it computes, for one colouring col (Section 2.1):
 *   M(v, {x}, {c})      = [col(v) == c]                               (base case)
 *   M(v, T_i, S)        = sum_{u in N(v)} sum_{S1 disjoint S2, S1 u S2 = S,
 *                          |S1| = |T_i'|, |S2| = |T_i''|}  M(v, T_i', S1) * M(u, T_i'', S2)
 *                                                                      (Eq. 1, d = 1)
 *   maps                = sum_v M(v, T, {all k colours})                (Eq. 3 sum)
 * where T_i is split by cutting one edge at its root: T_i' keeps the root and
 * T_i'' is the subtree hanging from the cut child (Section 2.1).  With d = 1
 * the DP counts labelled colourful maps (injective, edge-preserving, all k
 * colours distinct); the number of colourful copies is maps / |Aut(T)|.
 *
 * Arithmetic is exact modulo 2^256 (four 64-bit limbs, little-endian); a count
 * below 2^256 is therefore exact, and any larger count is its residue.
 *
 * Colouring (Algorithm 1, "pick a colour uniformly at random"): the paper
 * names no generator, so both sides implement the same counter-based rule:
 *   F(x) = SplitMix64 output function applied to the state x + 0x9E3779B97F4A7C15
 *          (Steele, Lea and Flood, OOPSLA 2014; Vigna's splitmix64.c)
 *   h    = F(F(F(seed) + j) + id(v))
 *   col  = floor(h * k / 2^64)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t w[4]; } u256;
typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- integers */

static void u256_add_to(u256 *acc, const u256 *x)
{
    u128 carry = 0;
    for (int i = 0; i < 4; i++) {
        u128 s = (u128)acc->w[i] + x->w[i] + carry;
        acc->w[i] = (uint64_t)s;
        carry = s >> 64;
    }
}

/* r = a * b mod 2^256, schoolbook on 64-bit limbs. */
static void u256_mul(u256 *r, const u256 *a, const u256 *b)
{
    uint64_t out[4] = {0, 0, 0, 0};
    if ((a->w[1] | a->w[2] | a->w[3] | b->w[1] | b->w[2] | b->w[3]) == 0) {
        u128 t = (u128)a->w[0] * b->w[0];           /* both operands below 2^64 */
        r->w[0] = (uint64_t)t; r->w[1] = (uint64_t)(t >> 64); r->w[2] = 0; r->w[3] = 0;
        return;
    }
    for (int i = 0; i < 4; i++) {
        if (a->w[i] == 0) continue;
        u128 carry = 0;
        for (int j = 0; i + j < 4; j++) {
            u128 t = (u128)a->w[i] * b->w[j] + out[i + j] + carry;
            out[i + j] = (uint64_t)t;
            carry = t >> 64;
        }
    }
    memcpy(r->w, out, sizeof out);
}

static int u256_is_zero(const u256 *x)
{
    return (x->w[0] | x->w[1] | x->w[2] | x->w[3]) == 0;
}

/* Exported for the test-suite (checked against Python integers). */
void cco_u256_mul(const uint64_t *a, const uint64_t *b, uint64_t *r)
{
    u256 x, y, z;
    memcpy(x.w, a, 32); memcpy(y.w, b, 32);
    u256_mul(&z, &x, &y);
    memcpy(r, z.w, 32);
}

void cco_u256_add(const uint64_t *a, const uint64_t *b, uint64_t *r)
{
    u256 x, y;
    memcpy(x.w, a, 32); memcpy(y.w, b, 32);
    u256_add_to(&x, &y);
    memcpy(r, x.w, 32);
}

/* ---------------------------------------------------------------- colouring */

static uint64_t splitmix64_out(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t cco_splitmix64(uint64_t state) { return splitmix64_out(state); }

int cco_colour(uint64_t seed, uint64_t j, uint64_t id, int k)
{
    uint64_t h = splitmix64_out(splitmix64_out(splitmix64_out(seed) + j) + id);
    return (int)(((u128)h * (uint64_t)k) >> 64);
}

static int popcount16(unsigned x) { int c = 0; while (x) { c += x & 1; x >>= 1; } return c; }

/* ---------------------------------------------------------------- template */

#define MAXK 16

typedef struct {
    int k;
    int nadj[MAXK];
    int adj[MAXK][MAXK];
} tmpl_t;

/* 0 = ok, -1 = not a tree / bad input. */
static int tmpl_build(tmpl_t *t, int k, const int32_t *edges)
{
    if (k < 1 || k > MAXK) return -1;
    memset(t, 0, sizeof *t);
    t->k = k;
    for (int e = 0; e < k - 1; e++) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return -1;
        for (int i = 0; i < t->nadj[a]; i++)
            if (t->adj[a][i] == b) return -1;
        t->adj[a][t->nadj[a]++] = b;
        t->adj[b][t->nadj[b]++] = a;
    }
    /* connected? (k-1 edges + connected = tree) */
    int seen[MAXK] = {0}, stack[MAXK], sp = 0, cnt = 0;
    stack[sp++] = 0; seen[0] = 1;
    while (sp) {
        int x = stack[--sp]; cnt++;
        for (int i = 0; i < t->nadj[x]; i++) {
            int y = t->adj[x][i];
            if (!seen[y]) { seen[y] = 1; stack[sp++] = y; }
        }
    }
    return cnt == k ? 0 : -1;
}

/*
 * |Aut(T)|: number of bijections p of V_T with {p(a), p(b)} an edge for every
 * edge {a, b}.  Backtracking over vertices in BFS order from vertex 0; every
 * tree edge joins a vertex to its BFS parent, so checking each vertex against
 * its parent checks every edge, and an injective edge map of a finite edge set
 * into itself is onto.  Each automorphism is enumerated, so the cost grows
 * with |Aut(T)| (fine for the workload templates; a k-star has (k-1)!).
 */
static int is_adj(const tmpl_t *t, int a, int b)
{
    for (int i = 0; i < t->nadj[a]; i++)
        if (t->adj[a][i] == b) return 1;
    return 0;
}

/* lab (optional): vertex labels; an automorphism must then map every vertex
 * to one with the same label. */
static int64_t aut_rec(const tmpl_t *t, const uint8_t *lab, const int *order, const int *par, int i,
                       int *img, int *used)
{
    if (i == t->k) return 1;
    int x = order[i];
    int64_t total = 0;
    for (int y = 0; y < t->k; y++) {
        if (used[y] || t->nadj[y] != t->nadj[x]) continue;
        if (lab && lab[y] != lab[x]) continue;
        if (par[x] >= 0 && !is_adj(t, img[par[x]], y)) continue;
        used[y] = 1; img[x] = y;
        total += aut_rec(t, lab, order, par, i + 1, img, used);
        used[y] = 0;
    }
    return total;
}

static int64_t automorphisms(int k, const int32_t *edges, const uint8_t *labels)
{
    tmpl_t t;
    if (tmpl_build(&t, k, edges)) return -1;
    int order[MAXK], par[MAXK], seen[MAXK] = {0}, head = 0, tail = 0;
    order[tail++] = 0; seen[0] = 1; par[0] = -1;
    while (head < tail) {
        int x = order[head++];
        for (int i = 0; i < t.nadj[x]; i++) {
            int y = t.adj[x][i];
            if (!seen[y]) { seen[y] = 1; par[y] = x; order[tail++] = y; }
        }
    }
    int img[MAXK], used[MAXK] = {0};
    return aut_rec(&t, labels, order, par, 0, img, used);
}

int64_t cco_automorphisms(int k, const int32_t *edges) { return automorphisms(k, edges, NULL); }

/* Label-preserving automorphisms of a vertex-labelled tree. */
int64_t cco_automorphisms_labelled(int k, const int32_t *edges, const uint8_t *labels)
{
    return labels ? automorphisms(k, edges, labels) : -1;
}

/* ---------------------------------------------------------------- colour sets */

/*
 * Colour sets are bitmasks over {0..k-1}.  The tables are indexed by the
 * position of a mask among all masks of the same size, listed in increasing
 * numeric order.  Both directions are filled by plain enumeration.
 */
typedef struct {
    int k;
    int *index_of;          /* [2^k] position of mask among masks of its size */
    int *masks[MAXK + 1];   /* masks[s][i] = i-th mask of size s */
    int count[MAXK + 1];    /* number of masks of size s = C(k, s) */
} sets_t;


static int sets_init(sets_t *s, int k)
{
    memset(s, 0, sizeof *s);
    s->k = k;
    int full = 1 << k;
    s->index_of = (int *)malloc(sizeof(int) * (size_t)full);
    if (!s->index_of) return -1;
    for (int z = 0; z <= k; z++) s->count[z] = 0;
    for (int mask = 0; mask < full; mask++) s->index_of[mask] = s->count[popcount16((unsigned)mask)]++;
    for (int z = 0; z <= k; z++) {
        s->masks[z] = (int *)malloc(sizeof(int) * (size_t)s->count[z]);
        if (!s->masks[z]) return -1;
    }
    int fill[MAXK + 1] = {0};
    for (int mask = 0; mask < full; mask++) {
        int z = popcount16((unsigned)mask);
        s->masks[z][fill[z]++] = mask;
    }
    return 0;
}

static void sets_free(sets_t *s)
{
    free(s->index_of);
    for (int z = 0; z <= MAXK; z++) free(s->masks[z]);
}

/* ---------------------------------------------------------------- the DP */

typedef struct {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const uint8_t *col;     /* colour of each vertex */
    const uint8_t *glab;    /* vertex labels of the graph and of the template */
    const uint8_t *tlab;    /*   (both NULL: unlabelled) */
    tmpl_t t;
    sets_t sets;
    int children[MAXK][MAXK];
    int nchildren[MAXK];
    int size[MAXK];         /* vertices in the subtree hanging from x */
    int failed;
} dp_t;

/* table for a partial tree of `sz` template vertices: n rows of C(k, sz) values */
static u256 *table_alloc(dp_t *d, int sz)
{
    size_t cells = (size_t)d->n * (size_t)d->sets.count[sz];
    u256 *p = (u256 *)calloc(cells ? cells : 1, sizeof(u256));
    if (!p) d->failed = 1;
    return p;
}

static void root_tree(dp_t *d, int x, int parent)
{
    d->nchildren[x] = 0;
    d->size[x] = 1;
    /* children in ascending vertex order */
    for (int y = 0; y < d->t.k; y++) {
        if (y == parent || !is_adj(&d->t, x, y)) continue;
        d->children[x][d->nchildren[x]++] = y;
        root_tree(d, y, x);
        d->size[x] += d->size[y];
    }
}

/*
 * Returns the table M(., T_x, .) of the whole subtree hanging from template
 * vertex x.  Starting from the single vertex x, the children of x are attached
 * one at a time; each attachment is one application of Eq. 1 with
 * T_i' = the part built so far (rooted at x) and T_i'' = the child's subtree.
 */
static u256 *subtree_table(dp_t *d, int x)
{
    /* base case: M(v, {x}, {c}) = [col(v) == c], times [label(v) == label(x)]
       for labelled counts (a map must preserve labels) */
    u256 *cur = table_alloc(d, 1);
    if (!cur) return NULL;
    const int c1 = d->sets.count[1];
    for (int64_t v = 0; v < d->n; v++)
        if (!d->glab || d->glab[v] == d->tlab[x])
            cur[(size_t)v * c1 + d->sets.index_of[1 << d->col[v]]].w[0] = 1;
    int cur_size = 1;

    for (int ci = 0; ci < d->nchildren[x]; ci++) {
        int c = d->children[x][ci];
        u256 *child = subtree_table(d, c);
        if (!child) { free(cur); return NULL; }
        const int a = cur_size, p = d->size[c], h = a + p;
        const int na = d->sets.count[a], np = d->sets.count[p], nh = d->sets.count[h];
        u256 *next = table_alloc(d, h);
        if (!next) { free(cur); free(child); return NULL; }

        /* positions of the non-zero entries of each child row (zero terms add nothing) */
        int64_t *nz_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d->n + 1));
        int64_t nnz = 0;
        if (!nz_ptr) { d->failed = 1; free(cur); free(child); free(next); return NULL; }
        for (int64_t u = 0; u < d->n; u++) {
            nz_ptr[u] = nnz;
            for (int i2 = 0; i2 < np; i2++) nnz += !u256_is_zero(&child[(size_t)u * np + i2]);
        }
        nz_ptr[d->n] = nnz;
        int *nz_idx = (int *)malloc(sizeof(int) * (size_t)(nnz ? nnz : 1));
        if (!nz_idx) { d->failed = 1; free(nz_ptr); free(cur); free(child); free(next); return NULL; }
        for (int64_t u = 0, q = 0; u < d->n; u++)
            for (int i2 = 0; i2 < np; i2++)
                if (!u256_is_zero(&child[(size_t)u * np + i2])) nz_idx[q++] = i2;

        for (int64_t v = 0; v < d->n; v++) {
            const u256 *cv = cur + (size_t)v * na;
            u256 *out = next + (size_t)v * nh;
            for (int64_t e = d->row_ptr[v]; e < d->row_ptr[v + 1]; e++) {     /* sum over u in N(v) */
                int64_t u = d->col_idx[e];
                const u256 *cu = child + (size_t)u * np;
                for (int i1 = 0; i1 < na; i1++) {                                /* S1, |S1| = |T_i'|  */
                    if (u256_is_zero(&cv[i1])) continue;
                    int s1 = d->sets.masks[a][i1];
                    for (int64_t q = nz_ptr[u]; q < nz_ptr[u + 1]; q++) {        /* S2, |S2| = |T_i''| */
                        int i2 = nz_idx[q];
                        int s2 = d->sets.masks[p][i2];
                        if (s1 & s2) continue;                                   /* S1, S2 disjoint    */
                        u256 prod;
                        u256_mul(&prod, &cv[i1], &cu[i2]);
                        u256_add_to(&out[d->sets.index_of[s1 | s2]], &prod);     /* into S = S1 u S2   */
                    }
                }
            }
        }
        free(nz_ptr);
        free(nz_idx);
        free(cur);
        free(child);
        cur = next;
        cur_size = h;
    }
    return cur;
}

/*
 * Counts labelled colourful maps of the template into the graph for one
 * colouring.
 *   n, row_ptr[n+1], col_idx[row_ptr[n]]: symmetric CSR (both directions).
 *   ids: optional [n] ids fed to the colouring rule (NULL = vertex index);
 *        lets a test run the oracle on an induced subgraph while keeping the
 *        colours of the original graph.
 *   colours: optional [n] explicit colours in [0, k) (overrides seed/j/ids).
 *   k, edges[2(k-1)]: the tree template; root: its root vertex.
 *   total[4]: sum_v M(v, T, all colours), mod 2^256.
 *   per_vertex: optional [n][4], M(v, T, all colours) for every v.
 *   glabels[n], tlabels[k]: optional vertex labels of the graph and the
 *        template (both or neither); a counted map then sends every template
 *        vertex to a graph vertex with the same label.
 * Returns 0, -1 for a bad template, root or label pair, -2 for an
 * out-of-range colour, -3 if memory ran out.
 */
int cco_count(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
              const int64_t *ids, const uint8_t *colours,
              int k, const int32_t *edges, int root,
              uint64_t seed, uint64_t j,
              uint64_t *total, uint64_t *per_vertex,
              const uint8_t *glabels, const uint8_t *tlabels)
{
    dp_t d;
    memset(&d, 0, sizeof d);
    if (tmpl_build(&d.t, k, edges)) return -1;
    if (root < 0 || root >= k) return -1;
    if (!glabels != !tlabels) return -1;
    d.glab = glabels;
    d.tlab = tlabels;
    d.n = n; d.row_ptr = row_ptr; d.col_idx = col_idx;
    uint8_t *col = (uint8_t *)malloc(n ? (size_t)n : 1);
    if (!col) return -3;
    for (int64_t v = 0; v < n; v++) {
        if (colours) {
            if (colours[v] >= k) { free(col); return -2; }
            col[v] = colours[v];
        } else {
            col[v] = (uint8_t)cco_colour(seed, j, ids ? (uint64_t)ids[v] : (uint64_t)v, k);
        }
    }
    d.col = col;
    if (sets_init(&d.sets, k)) { free(col); sets_free(&d.sets); return -3; }
    root_tree(&d, root, -1);
    u256 *top = subtree_table(&d, root);
    int rc = 0;
    if (!top) {
        rc = -3;
    } else {
        u256 acc = {{0, 0, 0, 0}};
        /* |T| = k, so the table has C(k, k) = 1 column: the full colour set */
        for (int64_t v = 0; v < n; v++) {
            u256_add_to(&acc, &top[v]);
            if (per_vertex) memcpy(per_vertex + 4 * (size_t)v, top[v].w, 32);
        }
        memcpy(total, acc.w, 32);
        free(top);
    }
    sets_free(&d.sets);
    free(col);
    return rc;
}
