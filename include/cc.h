/*
 * cc.h -- C ABI of the GB300 colour-coding tree counter.
 *
 * Method: arXiv 1804.09764 ("High-Performance Massive Subgraph Counting using
 * Pipelined Adaptive-Group Communication"), Section 2.1.  For a tree template
 * T on k vertices and a graph G, each colouring j assigns every vertex a colour
 * in [0, k) (Algorithm 1), and the dynamic program of Eq. 1 counts colourful
 * embeddings bottom-up over the partition tree of T; Eq. 3 scales the count by
 * k^k / k! into an estimate of the number of non-induced copies of T in G
 * (Section 2, "Subgraph-counting problem").
 *
 * Beyond one count (cc_count, cc_count_ex): several templates over the same
 * colourings with shared sub-tables (cc_count_multi), Algorithm 1 end to end
 * for a (1 +- epsilon, delta) estimate (cc_iterations_for, cc_estimate),
 * vertex-labelled templates (cc_template_load_labelled, cc_graph_set_labels),
 * a continuous-batching serving loop (cc_submit .. cc_serve_stats_get), and
 * the table gather on its own (cc_table_gather, cc_table_gather_noalloc).
 *
 * Conventions shared by every entry point:
 *   - Every call returns a cc_status: CC_OK (0), CC_PENDING (1, serving only)
 *     or a negative error.  On error, cc_last_error() returns a message for the
 *     calling thread; outputs are left unspecified.
 *   - The library copies every input it keeps; caller buffers may be freed as
 *     soon as a call returns.  Outputs go only into caller-owned buffers.
 *   - Handles (graphs, templates, requests) are owned by their context and die
 *     with it.
 *   - Wide integers are arrays of 64-bit limbs, least significant first.
 *   - All device work runs in this library's CUDA kernels on one GPU; there is
 *     no CPU fallback.
 *   - A context may be used from several threads; calls are serialised on an
 *     internal lock (the serving loop runs on its own thread).
 */
#ifndef CC_H
#define CC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cc_status;

#define CC_OK                0
#define CC_PENDING           1   /* serving: request not finished yet */
#define CC_ERR_INVALID_ARG  -1   /* null pointer, bad size, bad option */
#define CC_ERR_BAD_GRAPH    -2   /* self-loop, duplicate, asymmetric edge, index out of range */
#define CC_ERR_NOT_TREE     -3   /* template edges do not form a tree on 0..k-1 */
#define CC_ERR_K_RANGE      -4   /* k outside 1..16 */
#define CC_ERR_BUDGET       -5   /* the plan does not fit the HBM budget */
#define CC_ERR_WIDTH        -6   /* exact counts would need more than 256 bits */
#define CC_ERR_CUDA         -7   /* a CUDA call failed (message names it) */
#define CC_ERR_TIMEOUT      -8   /* a wait ran out of time */
#define CC_ERR_CANCELLED    -9   /* request was cancelled */
#define CC_ERR_NOT_FOUND   -10   /* unknown handle */
#define CC_ERR_CAPACITY    -11   /* caller buffer too small (needed size reported) */
#define CC_ERR_NO_MEMORY   -12   /* host allocation failed */
#define CC_ERR_INTERNAL    -13

typedef struct cc_ctx cc_ctx;
typedef int64_t cc_graph_id;
typedef int64_t cc_template_id;
typedef int64_t cc_req_id;

/* Context options.  Call cc_default_options() first, then change fields. */
typedef struct cc_options {
    int32_t device;            /* CUDA device ordinal */
    int32_t width_bits;        /* 0: exact counts, integer width chosen per table from a
                                  homomorphism bound; 64/128/192/256: every table at this
                                  width, counts returned as residues mod 2^width_bits */
    void *stream;              /* cudaStream_t for cc_count; NULL: the library makes one */
    void *arena;               /* caller-owned device memory that holds every library
                                  buffer (graphs, tables, scratch); NULL: the library
                                  allocates hbm_budget_bytes itself */
    uint64_t hbm_budget_bytes; /* size of arena; with arena == NULL, 0 means 90% of the
                                  device memory free at cc_create */
    int32_t split_threshold;   /* neighbour-list task size s (Algorithm 4); 0: default 4096 */
    int32_t batch;             /* colourings processed together in one pass; 0: largest
                                  that fits the budget, at most 16 */
    int32_t block_vertices;    /* vertices per streamed block; 0: largest that fits */
    int32_t use_cuda_graph;    /* 1: capture the per-batch schedule once and replay it */
    int32_t fused;             /* 1 (default): steps that attach a subtree to a single root
                                  vertex (a = 1) run the gather and the combine as one kernel
                                  whose neighbour sums go straight into the output row */
    int32_t autotune;          /* 1: autotuner.  On the first count of a (graph, template)
                                  it times the plan's shape, by coordinate descent over the
                                  options left at 0: split_threshold (1024, 4096, 16384),
                                  col_chunks (default rule, 1, 4, 16) and block_vertices
                                  (largest block that fits, 1/2, 1/4); each candidate runs
                                  one untimed pass, then the median of three timed passes
                                  decides.  On the first pass of every plan, each gather site
                                  times its kernel variants (gather_mode values, rows in
                                  flight) and keeps the fastest. */
    int32_t max_slots;         /* serving: groups (graph, template class) in flight at once (default 4) */
    int32_t timing;            /* 1: record per-kernel CUDA-event times (cc_kernel_stats) */
    int32_t gather_mode;       /* table-gather kernel: 1 (default): warp per row, persistent
                                  warps pulling rows from a counter, 4 neighbour rows in
                                  flight; 6: as 1 with 2 rows in flight; 5: warp per row, one
                                  pass (no counter); 0: bulk-copy (TMA) ring for rows of
                                  >= 1 KiB of 1- or 2-limb values; 2: warp per row, 16-byte
                                  vectors; 3: 32..256 threads per row; 4: as 6 plus whole-row
                                  L2 prefetch.  With autotune = 1 each gather site picks the
                                  fastest. */
    int32_t vertex_order;      /* 0 (default): active vertices numbered by decreasing degree
                                  (hub rows contiguous); 1: input order */
    int32_t col_chunks;        /* column segments per neighbour row in the persistent gathers
                                  (segment-major work order, so hub rows' segments are reused
                                  from L2).  0 (default): one 128-value warp sweep per segment
                                  (at most 16) for the heavy-vertex task gathers and the
                                  unfused gathers, whole rows for the fused gather + select
                                  kernels; n > 0: n segments everywhere (1: whole rows) */
    int32_t l2_persist_mb;     /* MiB of L2 set aside (for this context) for the rows read
                                  most often: before each table gather the stream's access
                                  window covers the first l2_persist_mb MiB of the source
                                  table, where degree ordering puts the hub rows (persisting
                                  hits, streaming misses); 0 (default): no window */
    int32_t full_rows;         /* 0 (default): in passes of one colouring (batch 1, k <= 16,
                                  fewer than 2^27 active vertices) the table gathers load
                                  only the entries of a neighbour's row whose colour set
                                  holds that neighbour's colour -- the others are zero by
                                  Eq. 1, since the subtree's root is mapped to the
                                  neighbour -- using a per-pass array of one colour byte
                                  per adjacency entry; 1: every gather reads whole rows */
    int32_t reserved[1];
} cc_options;

void cc_default_options(cc_options *opt);

/* Create a context on opt->device.  *out receives the handle. */
cc_status cc_create(cc_ctx **out, const cc_options *opt);
cc_status cc_destroy(cc_ctx *ctx);

/* Thread-local message of the last failing call; never NULL. */
const char *cc_last_error(void);
const char *cc_status_string(cc_status s);

#define CC_VALIDATE 1u   /* check symmetry, duplicates, self-loops, index range (host, O(m log m)) */

/*
 * Load an undirected graph G(V, E) (Section 2) in CSR form.
 *   n           number of vertices, 0 <= n < 2^31
 *   row_ptr     [n+1] int64 offsets, row_ptr[0] = 0, non-decreasing
 *   col_idx     [row_ptr[n]] int32 neighbour ids; both directions of every
 *               edge must be present; N(v) must not contain v
 *   Pointers may be host or device memory (detected); the library copies.
 *   flags       CC_VALIDATE to check the conditions above (CC_ERR_BAD_GRAPH)
 * The device copy drops isolated vertices from the table domain (they belong
 * to no embedding of a template with k >= 2) and lives in the arena.
 */
cc_status cc_graph_load_csr(cc_ctx *ctx, int64_t n, const int64_t *row_ptr,
                            const int32_t *col_idx, uint32_t flags, cc_graph_id *out);
cc_status cc_graph_free(cc_ctx *ctx, cc_graph_id g);

/*
 * A batch of many graphs loaded as one: every DP launch of a count then covers
 * all of them (the batching of many small graphs into one launch; the paper
 * counts one graph at a time, and its Eq. 1 is local to a vertex's
 * neighbourhood, so the DP of a disjoint union is the DPs of its parts).
 *   member_off  host [n_graphs + 1]: member graph i is vertices
 *               member_off[i] .. member_off[i + 1] - 1 of the CSR; 0 = first,
 *               n = last, non-decreasing (empty members allowed)
 *   n, row_ptr, col_idx, flags as cc_graph_load_csr, for the disjoint union
 *               (vertex ids of the union)
 * Member i's colours are drawn from its vertices' ids within the member (the
 * union id minus member_off[i]), so colouring j of a member is the colouring
 * j it gets when loaded alone and its counts (cc_count_batch) are the counts
 * of loading it alone, bit for bit.  cc_count and the other entry points take
 * the batch as one graph: their counts are the sums over the members.
 * Errors: those of cc_graph_load_csr; CC_ERR_INVALID_ARG (bad offsets);
 * CC_ERR_BAD_GRAPH also when an edge joins two members (always checked).
 */
cc_status cc_graph_load_batch(cc_ctx *ctx, int32_t n_graphs, const int64_t *member_off, int64_t n,
                              const int64_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                              cc_graph_id *out);

/*
 * Load a tree template T (Section 2.1), k = |V_T| in 1..16.
 *   edges  [2*(k-1)] int32 vertex pairs on 0..k-1
 *   root   root rho(T) of the partition (any vertex gives the same counts,
 *          Section 2.1: the root "can be picked arbitrarily"); -1: the planner
 *          picks the root with the lowest modelled cost
 */
cc_status cc_template_load(cc_ctx *ctx, int32_t k, const int32_t *edges, int32_t root,
                           cc_template_id *out);
cc_status cc_template_free(cc_ctx *ctx, cc_template_id t);

/*
 * Labelled templates (the extension of colour coding to vertex-labelled
 * templates cited in the paper's related work): template vertex x carries
 * labels[x] (k bytes, copied), and a counted map must send every template
 * vertex to a graph vertex with the same label.  Copies divide by the
 * label-preserving automorphisms (cc_result.aut).  Counting a labelled
 * template needs graph labels (cc_graph_set_labels); otherwise
 * CC_ERR_INVALID_ARG.  Errors as cc_template_load; labels NULL: invalid.
 */
cc_status cc_template_load_labelled(cc_ctx *ctx, int32_t k, const int32_t *edges, const uint8_t *labels,
                                    int32_t root, cc_template_id *out);

/*
 * Vertex labels of a loaded graph: labels[v] for v in [0, n) in the numbering
 * of cc_graph_load_csr (host array, copied; NULL removes the labels).  Used
 * by labelled templates only; unlabelled templates ignore them.  Drops the
 * graph's cached plans.  Errors: CC_ERR_NOT_FOUND, CC_ERR_BUDGET,
 * CC_ERR_INVALID_ARG while a queued or running serving request uses the graph.
 */
cc_status cc_graph_set_labels(cc_ctx *ctx, cc_graph_id g, const uint8_t *labels);

/* Results of a count (one per call or per request). */
typedef struct cc_result {
    int32_t k;
    int32_t limbs;          /* 64-bit limbs per count needed/written */
    int32_t exact;          /* 1: counts are exact colourful copies (maps / |Aut T|);
                               0: residues of labelled maps mod 2^(64*limbs) */
    int32_t n_iter;
    int64_t aut;            /* |Aut(T)| */
    int32_t root;           /* partition root used */
    int32_t batch;          /* colourings per pass used */
    double estimate;        /* mean over colourings of copies_j * k^k / k! (Eq. 3); exact mode */
    double median_of_means; /* Algorithm 1's final step over t groups; exact mode */
    double device_seconds;  /* GPU time of the colourings (CUDA events) */
    double wall_seconds;    /* host wall time of the call / request latency */
    uint64_t workspace_bytes; /* device bytes the plan used (tables + scratch) */
    int64_t kernel_launches;  /* kernels launched for this call */
} cc_result;

/*
 * Run colourings 0..n_iter-1 from `seed` (Algorithm 1's outer loop).
 *   counts  [n_iter][limbs_capacity] uint64, host memory: per-colouring
 *           colourful copies (exact mode) or map residues (forced width)
 *   limbs_capacity must be >= res->limbs (CC_ERR_CAPACITY otherwise; res->limbs
 *           then says how many are needed)
 *   res     optional (may be NULL)
 * Colour of vertex v in colouring j: h = F(F(F(seed) + j) + v),
 * col = floor(h * k / 2^64), F = SplitMix64 output function of state x + 0x9E3779B97F4A7C15.
 */
cc_status cc_count(cc_ctx *ctx, cc_graph_id g, cc_template_id t, uint64_t seed, int32_t n_iter,
                   uint64_t *counts, int32_t limbs_capacity, cc_result *res);

/* Extended arguments for cc_count_ex. */
typedef struct cc_count_args {
    uint64_t seed;
    int64_t first_iter;              /* index j of the first colouring */
    int32_t n_iter;
    int32_t mom_groups;              /* t for the median of means (0 -> 1) */
    int32_t width_bits;              /* -1: context default; otherwise as cc_options.width_bits */
    int32_t reserved0;
    const int64_t *sample_vertices;  /* optional host [n_sample] original vertex ids */
    int64_t n_sample;
    uint64_t *sample_maps;           /* optional host [n_iter][n_sample][limbs_capacity]:
                                        M(v, T, all colours) = labelled colourful maps with the
                                        root on v, mod 2^(64*limbs) */
    uint64_t *maps;                  /* optional host [n_iter][limbs_capacity]: labelled maps
                                        (sum over v, before the division by |Aut T|) */
} cc_count_args;

cc_status cc_count_ex(cc_ctx *ctx, cc_graph_id g, cc_template_id t, const cc_count_args *args,
                      uint64_t *counts, int32_t limbs_capacity, cc_result *res);

/*
 * cc_count_ex per member graph of a batch (cc_graph_load_batch; a graph loaded
 * by cc_graph_load_csr is a batch of one).  One pass of the DP covers every
 * member; only the root sums are kept per member.
 *   counts     host [n_graphs][n_iter][limbs_capacity]: member i's colourful
 *              copies (Eq. 3's numerator) per colouring, as cc_count_ex
 *   estimates  optional host [n_graphs]: member i's estimate (Eq. 3, mean
 *              over the colourings)
 *   args       as cc_count_ex; args->maps, if set, is [n_graphs][n_iter][cap];
 *              sample_maps as cc_count_ex (union ids)
 *   res        the fields shared by the members; estimate and median_of_means
 *              hold the batch's total estimate (the sum over members)
 * Errors as cc_count_ex.
 */
cc_status cc_count_batch(cc_ctx *ctx, cc_graph_id g, cc_template_id t, const cc_count_args *args,
                         uint64_t *counts, int32_t limbs_capacity, double *estimates, cc_result *res);

/* Member graphs of a loaded graph (1 unless loaded by cc_graph_load_batch). */
cc_status cc_graph_members(cc_ctx *ctx, cc_graph_id g, int32_t *n_graphs);

/* Static description of the plan for (graph, template) under the context options. */
typedef struct cc_plan_info {
    int32_t k, root, n_chains, n_tables;
    int32_t limbs_root;              /* width of the root chain in 64-bit limbs */
    int32_t batch;                   /* colourings per pass */
    int64_t n_vertices, n_active, n_directed_edges;
    int64_t n_blocks;                /* vertex blocks per chain */
    double updates_per_colouring;    /* sum over gathered non-leaf passive tables of 2m*C(k,p) */
    double gather_bytes_per_colouring;   /* algorithmic bytes of the table gathers */
    double algorithmic_bytes_per_colouring; /* gathers + table writes + CSR + leaf colour reads */
    double pairs_per_colouring;      /* combine multiply-adds per colouring */
    uint64_t workspace_bytes;
    int64_t table4_memory, table4_computation;  /* Table 4 cost numbers of the partition */
    double limb_products_per_colouring;  /* 64-bit limb multiplications of the general combines
                                            (a >= 2, p >= 2) at their widths, over every output
                                            of Eq. 1: per product of an La-limb by an Lb-limb
                                            value into L limbs, the limb pairs i + j < L (low
                                            halves) and i + j + 1 < L (high halves).  (The
                                            kernels compute only the outputs whose colour set
                                            holds the vertex's own colour, h/k of a step's.) */
    int64_t split_threshold;         /* neighbour-list task size s in use (Algorithm 4) */
    int64_t block_vertices;          /* vertices per streamed block in use */
    int32_t col_chunks;              /* column segments in use (cc_options.col_chunks meaning) */
    int32_t shape_tuned;             /* 1: split, segments and block size come from the autotuner */
    /* the device memory the same plan would need (at the same batch) if no
       count table were freed before the end of the pass, if the vertices were
       not streamed in blocks, and with neither: the one-GPU counterpart of the
       paper's peak-memory comparison (Section 4.4) of its pipelined schedule (Section 3.2) */
    uint64_t workspace_no_reuse_bytes, workspace_no_blocks_bytes, workspace_naive_bytes;
} cc_plan_info;

/* Describes the plan the last cc_count of (g, t) used while it is still
 * cached, else plans a count of opt.batch (default 16) colourings. */
cc_status cc_plan_info_get(cc_ctx *ctx, cc_graph_id g, cc_template_id t, cc_plan_info *out);

/*
 * The steps of a plan: one row per application of Eq. 1 (Section 2.1), i.e.
 * per child attached to a chain (chains in post-order, the root chain last),
 * with the integer widths the homomorphism bounds gave it and how the last
 * pass ran it for the light vertices (those with at most split_threshold
 * neighbours) of the first vertex block.  Describes the cached plan of the
 * last count of (g, t) under the context's width policy; with no such plan
 * (or a plan that has not run) every path is CC_PATH_NOT_RUN.
 *   out[cap] receives min(cap, steps) rows; *n_steps the number of steps.
 * Errors: CC_ERR_INVALID_ARG (NULL ctx or n_steps, cap < 0), CC_ERR_NOT_FOUND.
 */
#define CC_PATH_NOT_RUN        0
#define CC_PATH_CHAIN_KERNEL   1  /* gather + a = 1 combine, and in the same kernel the chain's p = 1 steps */
#define CC_PATH_IN_CHAIN       2  /* a p = 1 step run inside the chain kernel of its chain's first step */
#define CC_PATH_SEGMENTED      3  /* column-segmented gather + a = 1 combine, then the leaf-chain kernel */
#define CC_PATH_FUSED_SELECT   4  /* gather + a = 1 combine in one kernel */
#define CC_PATH_GATHER_SELECT  5  /* table gather kernel, then the a = 1 combine */
#define CC_PATH_GATHER_COMBINE 6  /* table gather kernel, then the general combine */
#define CC_PATH_LEAF_SELECT    7  /* a = 1 step attaching a leaf: select from the colour histogram */
#define CC_PATH_LEAF_COMBINE   8  /* p = 1 step: combine with the colour histogram */
typedef struct cc_step_info {
    int32_t chain, step;     /* chain index, step within the chain */
    int32_t vertex;          /* template vertex the chain is rooted at */
    int32_t child;           /* template vertex whose subtree this step attaches */
    int32_t h, a, p;         /* |T_i|, |T_i'|, |T_i''| */
    int32_t src_chain;       /* chain whose table is gathered; -1 for a leaf child */
    int32_t is_root;         /* 1 for the root chain */
    int32_t limbs;           /* 64-bit limbs the step's own bound needs */
    int32_t agg_limbs;       /* limbs of its neighbour sums */
    int32_t src_limbs;       /* limbs of the gathered table (0 for a leaf child) */
    int32_t chain_limbs;     /* limbs of the chain's table (root chain: of the totals) */
    int32_t path;            /* CC_PATH_* */
    int32_t kernel_limbs[3]; /* limb template arguments of that path's kernel:
                                chain kernel <Ls, Lf, Ld>; fused select <Ls, -, Ld>;
                                gather + combine <Ls, Lagg, Lout>; leaf paths <Lin, -, Lout> */
} cc_step_info;

cc_status cc_plan_steps_get(cc_ctx *ctx, cc_graph_id g, cc_template_id t, cc_step_info *out, int32_t cap,
                            int32_t *n_steps);

/* Per-kernel CUDA-event statistics (opt.timing = 1); cumulative since reset.
 * Kinds, in order: colour; hist (colour histograms of N(v), the leaf gather);
 * gather (table gather of vertices with at most split_threshold neighbours);
 * combine (general Eq. 1 combine); reduce (root sum); fused (table gather +
 * a = 1 combine, with the leaf steps that follow it in the chain, for those
 * vertices); select (a = 1 combine); combine_hist (p = 1 combine); heavy
 * (vertices with more neighbours: Algorithm 4 sub-list tasks, their partial-row
 * sums and the combines that follow them in a fused step). */
#define CC_KERNEL_KINDS 9
typedef struct cc_kernel_stats {
    const char *name[CC_KERNEL_KINDS];
    int64_t launches[CC_KERNEL_KINDS];
    double seconds[CC_KERNEL_KINDS];   /* summed event durations */
    double bytes[CC_KERNEL_KINDS];     /* algorithmic bytes moved */
    int64_t total_launches;            /* every kernel launched by the library */
} cc_kernel_stats;

cc_status cc_kernel_stats_get(cc_ctx *ctx, cc_kernel_stats *out);
cc_status cc_kernel_stats_reset(cc_ctx *ctx);

/* Statistics per kernel instantiation since the last reset: one row per
 * (kind, instantiation) launched, sorted by kind then name.  The name carries
 * the limb template arguments, e.g. "gather_select_chain_kernel<2,2,3>".
 * Launches are always counted; seconds, bytes and timed_launches (opt.timing
 * = 1) cover the timed groups of launches in which this instantiation was the
 * only kernel, so seconds / timed_launches is its average launch duration and
 * bytes / seconds its algorithmic rate.
 *   out[cap] receives min(cap, rows) rows; *n (optional) the number of rows.
 * Errors: CC_ERR_INVALID_ARG (NULL ctx, cap < 0, out NULL with cap > 0). */
typedef struct cc_instance_stats {
    char name[96];           /* NUL-terminated, truncated if longer */
    int32_t kind;            /* index into cc_kernel_stats */
    int32_t reserved;
    int64_t launches;
    int64_t timed_launches;
    double seconds;
    double bytes;
} cc_instance_stats;

cc_status cc_kernel_instance_stats_get(cc_ctx *ctx, cc_instance_stats *out, int32_t cap, int32_t *n);

/*
 * Eq. 1's neighbour sum for one count table on its own (the table-gather step):
 *   agg[v] = sum_{u in N(v)} X[u]   for every v in [0, n)
 * where a row holds `values` integers of `limbs` 64-bit limbs, added modulo
 * 2^(64*limbs).  All pointers are device memory:
 *   row_ptr [n+1] int64, col_idx [row_ptr[n]] int32 (any CSR, symmetric or not),
 *   X, agg  [n][values][limbs] uint64 (may not overlap).
 * Neighbour lists longer than split_threshold (0: 1024) are cut into tasks of at
 * most that many neighbours (Algorithm 4); the tasks' partial rows and the task
 * list are scratch carved from the context's arena and released before return.
 * Runs on the context's stream and synchronises it.
 * Errors: CC_ERR_INVALID_ARG (bad sizes, limbs outside 1..4), CC_ERR_BUDGET
 * (scratch does not fit the arena), CC_ERR_CUDA.
 */
cc_status cc_table_gather(cc_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                          const uint64_t *X, uint64_t *agg, int64_t values, int32_t limbs,
                          int32_t split_threshold);

/*
 * cc_table_gather without any device allocation.  The paper has no counterpart:
 * this is a library service for callers that cannot allocate device memory (a
 * framework that owns all device memory through its own pool, a latency-bound
 * loop where cudaMalloc/cudaFree and their implicit synchronisation are not
 * acceptable, a process with a fixed memory budget).
 *   Computes agg[v] = sum_{u in N(v)} X[u] exactly like cc_table_gather (same
 *   kernels, same results) with the same argument meaning; no context needed.
 *   All pointers are device memory on the calling thread's current device;
 *   stream is a cudaStream_t (NULL: the legacy default stream).
 *   Scratch: the task list and the tasks' partial rows live in a 64 MiB
 *   file-scope device array that every GPU loading this library holds until the
 *   process exits.  It fits at most (64 MiB - ~1.3 KiB) / (28 + values*limbs*8)
 *   split tasks; larger inputs return CC_ERR_CAPACITY before any gather kernel
 *   runs (raise split_threshold to need fewer tasks).
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) and caches it.
 *   Every call synchronises `stream` once, to read the task count back, and
 *   returns with the gather kernels queued on `stream`; because of that
 *   synchronisation and read-back no call can be captured into a CUDA graph.  All calls share the array and
 *   each call rewrites what it reads, so nothing needs clearing between calls,
 *   but calls whose kernels overlap on the GPU race on the array: serialise them.
 *   Calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: CC_ERR_INVALID_ARG (also for a decreasing row_ptr, found on the
 * device before any gather kernel runs), CC_ERR_CAPACITY, CC_ERR_CUDA.
 */
cc_status cc_table_gather_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                  const uint64_t *X, uint64_t *agg, int64_t values, int32_t limbs,
                                  int32_t split_threshold, void *stream);

/* ------------------------------------------------------------------ serving */

/* One count request (same arithmetic as cc_count_ex). */
typedef struct cc_request {
    cc_graph_id graph;
    cc_template_id tmpl;
    uint64_t seed;
    int64_t first_iter;
    int32_t n_iter;
    int32_t priority;       /* reserved */
} cc_request;

/*
 * Submit a request to the continuous-batching loop.  Admitted requests are
 * grouped by graph and by template up to isomorphism (isomorphic templates
 * have the same counts).  A group runs one colouring pass at a time on its own
 * stream; each pass takes the next pending colourings of all the group's
 * requests in arrival order, up to cc_options.batch (default 16), so one
 * launch carries colourings of several requests, and a request joins its
 * group's next pass as soon as it is admitted.  Up to max_slots groups run
 * concurrently; a request that needs a new group is admitted when a slot is
 * free and the group's workspace fits the free arena.  Results are those of
 * cc_count_ex with the request's seed, first_iter and n_iter.
 */
cc_status cc_submit(cc_ctx *ctx, const cc_request *req, cc_req_id *out);
/* CC_PENDING while running; CC_OK with results; an error if it failed.
 * counts as for cc_count.  A finished request is forgotten after a successful
 * poll/wait that returns its results. */
cc_status cc_poll(cc_ctx *ctx, cc_req_id id, cc_result *res, uint64_t *counts, int32_t limbs_capacity);
cc_status cc_wait(cc_ctx *ctx, cc_req_id id, int64_t timeout_ns, cc_result *res, uint64_t *counts,
                  int32_t limbs_capacity);
cc_status cc_cancel(cc_ctx *ctx, cc_req_id id);

typedef struct cc_serve_stats {
    int64_t submitted, completed, failed, cancelled, in_flight, queued;
    double p50_latency_s, p99_latency_s, mean_latency_s;
    double busy_seconds;           /* wall time with at least one request in flight */
    int64_t admissions_deferred;   /* times a queued request waited for memory or a slot */
    int64_t passes;                /* colouring passes run */
    int64_t shared_passes;         /* passes whose launches carried colourings of two or more requests */
    int64_t colourings_run;        /* colourings computed by those passes */
    int64_t groups;                /* groups (graph, template class) running now */
} cc_serve_stats;

cc_status cc_serve_stats_get(cc_ctx *ctx, cc_serve_stats *out);

/* ------------------------------------------------- several templates at once */

/*
 * Counts of n_tmpl templates with the same k over the same colourings (the
 * colourings of cc_count with args->seed, first_iter, n_iter).  The templates
 * are planned one by one (their requested roots, or the planner's) and merged:
 * a rooted subtree whose canonical form already occurs in an earlier template
 * reuses that table, and the colouring and colour histograms are computed once
 * per pass for all of them -- the shared sub-templates of graphlet-frequency
 * counting (Section 2.1: each table depends only on the rooted subtree T_i and
 * the colouring).  Results equal those of cc_count on each template.
 *   counts, args->maps: [n_tmpl][n_iter][limbs_capacity]; res: [n_tmpl] (or NULL;
 *   device_seconds and kernel_launches there are those of the shared passes).
 *   args->n_sample must be 0.  The merged plan is not cached.
 * Errors: as cc_count; CC_ERR_INVALID_ARG for n_tmpl < 1, different k, or
 * sampled vertices.
 */
cc_status cc_count_multi(cc_ctx *ctx, cc_graph_id g, const cc_template_id *tmpls, int32_t n_tmpl,
                         const cc_count_args *args, uint64_t *counts, int32_t limbs_capacity, cc_result *res);

typedef struct cc_multi_info {
    int32_t chains;                  /* tables (chains) of the merged plan */
    int32_t chains_separate;         /* their sum over the templates planned alone */
    double updates_per_colouring;    /* gathered edge x colour-set updates, merged */
    double updates_per_colouring_separate;
    uint64_t workspace_bytes;        /* merged plan, for n_iter colourings */
    int32_t batch;
    int32_t reserved;
} cc_multi_info;

/* Plans the merged count (as cc_count_multi with n_iter colourings) without
 * running it. */
cc_status cc_multi_plan_info_get(cc_ctx *ctx, cc_graph_id g, const cc_template_id *tmpls, int32_t n_tmpl,
                                 int32_t n_iter, cc_multi_info *out);

/* ------------------------------------------------- (epsilon, delta) driver */

/*
 * Algorithm 1's sample size, with the constants it leaves as O(.) fixed by the
 * following argument.  With N copies of T and p = k!/k^k, the colourful count
 * Y of one colouring satisfies 0 <= Y <= N and E[Y] = pN, so E[Y^2] <= N E[Y]
 * and X = Y/p (Eq. 3) has Var X / (E X)^2 <= 1/p - 1.  The mean of
 * s = ceil(4 (1/p - 1) / epsilon^2) colourings is then outside (1 +- epsilon) N
 * with probability <= 1/4 (Chebyshev), and the median of
 * t = ceil(8 ln(1/delta)) such means with probability <= exp(-t/8) <= delta
 * (Hoeffding on the number of failed groups).
 *   n_iter = s * t (at least 1 each), groups = t.  Host only, FP64.
 * Errors: CC_ERR_K_RANGE (k outside 1..16); CC_ERR_INVALID_ARG (NULL outputs,
 * epsilon <= 0, delta outside (0, 1), NaN); CC_ERR_CAPACITY (n_iter >= 2^62).
 */
cc_status cc_iterations_for(int32_t k, double epsilon, double delta, int64_t *n_iter, int32_t *groups);

typedef struct cc_estimate_result {
    int32_t k;
    int32_t groups;           /* t */
    int64_t n_iter;           /* colourings counted: groups * per_group */
    int64_t per_group;        /* s */
    double estimate;          /* median of the t group means of (k^k/k!) * copies_j */
    double mean;              /* mean over all colourings */
    double min_group_mean, max_group_mean;
    double device_seconds, wall_seconds;
} cc_estimate_result;

/*
 * Algorithm 1 end to end: colourings first_iter .. first_iter + n_iter - 1 of
 * `seed` (n_iter, t from cc_iterations_for), counted exactly as cc_count does
 * in chunks of at most 4096 colourings; colouring j belongs to group j / s.
 * max_iter > 0 refuses (CC_ERR_CAPACITY, nothing run) when n_iter would exceed
 * it.  Exact counts only (widths from the bound); errors as cc_count.
 */
cc_status cc_estimate(cc_ctx *ctx, cc_graph_id g, cc_template_id t, uint64_t seed, int64_t first_iter,
                      double epsilon, double delta, int64_t max_iter, cc_estimate_result *out);

/* ------------------------------------------------------------------ helpers */

/* Table 4 cost numbers of the partition of a template from a given root with
 * children attached largest subtree first (order = 0) or by the planner's own
 * order (order = 1).  Host only. */
cc_status cc_template_cost(int32_t k, const int32_t *edges, int32_t root, int32_t order,
                           int64_t *memory, int64_t *computation);

/* |Aut(T)| from rooted canonical forms at the tree centre.  Host only. */
cc_status cc_template_automorphisms(int32_t k, const int32_t *edges, int64_t *aut);

/* The label-preserving automorphisms of a vertex-labelled tree (labels[k]).
 * Host only. */
cc_status cc_template_automorphisms_labelled(int32_t k, const int32_t *edges, const uint8_t *labels, int64_t *aut);

/* Canonical form of a tree template (labels[k] or NULL): a NUL-terminated
 * string, equal for two templates exactly when they are isomorphic (by a
 * label-preserving map when labelled) -- the key by which the serving loop
 * lets requests of isomorphic templates share passes (isomorphic templates
 * have the same counts).  Written to out[cap]; CC_ERR_CAPACITY (nothing
 * written) when cap is below the form's length + 1.  Host only. */
cc_status cc_template_canonical_form(int32_t k, const int32_t *edges, const uint8_t *labels, char *out,
                                     int32_t cap);

/* The rate of 64-bit limb products (a 64 x 64-bit multiply's low and high
 * halves counted as two, each with its carry-propagating add) that the
 * context's GPU sustains on register operands: the arithmetic ceiling of the
 * general combine, whose work cc_plan_info counts in the same unit.  Runs two
 * short kernels (~10 ms) and synchronises the context's stream. */
cc_status cc_limb_product_rate(cc_ctx *ctx, double *per_second);

/* Library version string. */
const char *cc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CC_H */
