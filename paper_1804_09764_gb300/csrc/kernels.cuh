// kernels.cuh -- launch wrappers for the colour-coding DP kernels (sm_103a).
//
// Data layout in device memory (one "pass" processes B colourings at once):
//   colours  col[v * B + b]                       uint8
//   hist     hist[(v * B + b) * k + c]            uint32  (leaf gather, p = 1)
//   tables   X[((v * B + b) * Cs + s) * L + limb] uint64  (C(k, |T|) colex columns,
//                                                         row stride Cs = col_stride(C))
// v runs over the active (non-isolated) vertices in the library's compact
// numbering.  A "block" is a contiguous vertex range [v0, v1) whose working
// rows (aggregates, chain intermediates) are stored at local row v - v0.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace cc {

// Names of the kernel instantiations the launch wrappers below issued on the
// calling thread, e.g. "gather_select_chain_kernel<2,2,3>" (template limb
// arguments; -1 leaves one out).  take_launch_names() returns them and clears
// the list; the executor files them under the kernel kind being timed.
void note_launch(const char *kernel, int a = -1, int b = -1, int c = -1);
std::vector<std::string> take_launch_names();

struct ColourParams {
    uint64_t hj[64];  // F(F(seed) + j) for the colourings of the pass (b < B <= 64)
};

// per-pass parameters live in device memory so a captured graph can be replayed
void launch_colour(cudaStream_t st, int64_t n_act, int B, int k, const int64_t *orig_id,
                   const ColourParams *prm, uint8_t *col);

// labels (optional): count only neighbours u with labels[u] == want
void launch_hist(cudaStream_t st, int64_t v0, int64_t v1, int B, int k, const int64_t *row_ptr,
                 const int32_t *col_idx, const uint8_t *col, uint32_t *hist, const uint8_t *labels = nullptr,
                 int want = 0);

// labelled templates: rows[v][0 .. row_words) = 0 for v in [0, nv) with labels[v] != want
void launch_mask_rows(cudaStream_t st, int64_t nv, int64_t row_words, const uint8_t *labels, int want, uint64_t *rows);

// Entries that a gathered table holds as zero by construction: M(u, T, S) = 0
// when col(u) is not in S (the root of T is mapped to u, Eq. 1), so in a pass
// of one colouring (B = 1, row = the C(k, |T|) colex columns) a gather need not
// load them.  ncol[e] = col(col_idx[e]) (neighbour colours of the pass, one
// byte per list entry, written by launch_neighbour_colours); smask[s] = the
// colour set of column s as a bit mask (0 for the padding column).  With ncol
// == nullptr every entry is loaded.  Needs k <= 16 and ids below 2^27 (the
// colour travels in bits 27..30 of the id broadcast to the warp).
struct AbsentSkip {
    const uint8_t *ncol = nullptr;
    const uint16_t *smask = nullptr;
};

// ncol[e] = col[col_idx[e]] for e in [0, nnz) (one colouring per pass)
void launch_neighbour_colours(cudaStream_t st, int64_t nnz, const int32_t *col_idx, const uint8_t *col,
                              uint8_t *ncol);

// agg[v - v0] = sum_{u in N(v)} X[u]  over rows of R values; light vertices only
// (deg <= split), heavy ones go through tasks + reduce.
// prefetch: also request each neighbour row whole into L2 (cp.async.bulk.prefetch)
// next: zeroed device counter -> persistent grid whose warps pull items from it;
//       nullptr -> one warp per item
// nb: neighbour rows loaded before adding (2 or 4)
// nch, G (with next): work items are (column segment, G consecutive vertices),
// segment-major (see launch_gather_tasks)
void launch_gather_light(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                         const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X,
                         int64_t R, uint64_t *agg, bool prefetch = false, unsigned long long *next = nullptr,
                         int nb = 4, int nch = 1, int G = 1, AbsentSkip sk = {});

// tasks [t0, t1): neighbour sub-lists (task_v, task_e0, task_e1); each writes partial[t - t0]
// nch > 1 (with next): the row is split into nch column segments run
// segment-major, so hub rows' segments are reused from L2 by the warps in flight
void launch_gather_tasks(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1,
                         const int32_t *col_idx, const int64_t *task_e, const uint64_t *X,
                         int64_t R, uint64_t *partial, bool prefetch = false, unsigned long long *next = nullptr,
                         int nb = 4, int nch = 1, AbsentSkip sk = {});

// column segments for rows of R values of Ls limbs: requested > 0 as given
// (<= 64); 0: one 128-value warp sweep per segment, at most 16
int column_segments(int64_t R, int Ls, int requested);

// Vectorised warp versions (16-byte loads, several neighbours in flight) for
// rows of 1- or 2-limb values; usable when vec_gather_ok(Ls, R).
bool vec_gather_ok(int Ls, int64_t R);
void launch_gather_light_vec(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                             const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int64_t R,
                             uint64_t *agg);
void launch_gather_tasks_vec(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                             const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial);

// Group versions: 32..256 threads per row so the whole row is loaded in one
// pass (rows of 1- or 2-limb values; same condition as the vectorised kernels).
void launch_gather_light_group(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                               const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int64_t R,
                               uint64_t *agg);
void launch_gather_tasks_group(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                               const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial);

// Bulk-copy (TMA) versions of the two gathers above: persistent CTAs stream
// neighbour-row segments into shared memory through an mbarrier ring.  Usable
// when bulk_gather_ok(Ls, R).  *err receives a non-zero code if a wait timed out.
bool bulk_gather_ok(int Ls, int64_t R);
// once per process and device before the first launch (shared-memory opt-in)
void init_kernel_attributes();
void launch_gather_light_bulk(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                              const int64_t *row_ptr, const int32_t *col_idx, int64_t nnz, const uint64_t *X,
                              int64_t R, uint64_t *agg, int *err);
void launch_gather_tasks_bulk(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                              int64_t nnz, const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial,
                              int *err);

// heavy vertices [h0, h1) of the heavy list: agg[v - v0] = sum of their partial rows
void launch_gather_reduce(cudaStream_t st, int Ld, int64_t h0, int64_t h1, int64_t v0, int64_t t0,
                          const int32_t *heavy_v, const int64_t *heavy_tptr, const uint64_t *partial,
                          int64_t R, uint64_t *agg);

// combine kernels (Eq. 1 inner sum).  Rows: act C(k,a), agg C(k,p), out C(k,h)
// valid columns, stored with strides Cas, Cps, Chs (>= the column counts; extra
// output columns are written as zero); B rows per vertex.
// act rows of La-limb values, agg rows of Lb-limb values, out rows of L limbs
// (La, Lb <= L)
// cv: colours of the block's rows ([vertex][colouring]); rm_h: the rank table
// of size-h sets; elig: for each colour c the E = C(k-1, h-1) ranks of the
// h-sets holding c, increasing (only those outputs can be non-zero)
void launch_combine_generic(cudaStream_t st, int L, int La, int Lb, int64_t nv, int B, int64_t Ch, int64_t Chs,
                            int64_t Cas, int64_t Cps, int64_t npairs, const uint32_t *pairs, const uint64_t *act,
                            const uint64_t *agg, uint64_t *out, int k, const uint8_t *cv, const uint16_t *rm_h,
                            const uint16_t *elig, int64_t E);
// a = 1: act is the single vertex v with colour col(v)
void launch_combine_select(cudaStream_t st, int L, bool agg_is_hist, int64_t v0, int64_t nv, int B, int k,
                           int64_t Ch, int64_t Chs, int64_t Cps, const uint16_t *rm, const uint8_t *col,
                           const void *agg, uint64_t *out);
// 64-bit limb products per second that this GPU sustains in registers (the
// combines' multiply-add chains without their loads); synchronises st.
// scratch: one device word.  0 on a CUDA error.
double limb_product_rate(cudaStream_t st, uint64_t *scratch);

// p = 1: agg is the colour histogram of N(v); pairs = the (h, h-1) split table;
// act rows of La-limb values (La <= L)
void launch_combine_hist(cudaStream_t st, int L, int La, int64_t nv, int B, int k, int64_t Ch, int64_t Chs,
                         int64_t Cas, int h, const uint32_t *pairs, const uint64_t *act, const uint32_t *hist,
                         uint64_t *out, const uint8_t *cv, const uint16_t *rm_h, const uint16_t *elig, int64_t E);

// Fused table gather + a = 1 combine for the light vertices of [v0, v1) (persistent
// warps on the zeroed counter `next`): out[v][b][T u {col}] = sum_u X[u][b][T].
// add_p: (p -> p+1) add-a-colour ranks; rm_h: remove-a-colour ranks of size h.
void launch_gather_select(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                          const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int B, int k,
                          int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *add_p,
                          const uint16_t *rm_h, const uint8_t *col, uint64_t *out, unsigned long long *next,
                          int nb = 4, int nch = 1, int G = 1, int64_t out_vs = 0, AbsentSkip sk = {});
// (nch, G as for launch_gather_light; out_vs: 64-bit words between the output
// rows of consecutive vertices, 0 = B * Chs * Ld)
// Chain version: after the fused step the same warp runs the chain's following
// p = 1 steps (leaf children) for the vertex, out_j[S] = sum over c in S of
// out_{j-1}[S \ {c}] * hist[c].  The rows of vertex v for step j start at
// out[j] + (v - v0) * vs[j] (vs in 64-bit words, >= B * Chs[j] * Ld): steps that
// share a buffer give every vertex the same slot, so no warp writes into rows
// another warp has yet to read.  col and hist[j] are whole-graph arrays
// (indexed by global vertex id).
struct LeafChain {
    int n;                       // number of p = 1 steps after the fused step (<= 15)
    int h[15];
    int64_t Ch[15], Chs[15], vs[15];
    const uint32_t *pairs[15];   // (h, h-1) split tables (the heavy vertices' p = 1 kernels)
    const uint16_t *rm[15];      // rank of S \ {c} per (S, c) of size h, 0xFFFF when c is not in S
    const uint32_t *hist[15];    // colour histograms of the leaf's label (or of all neighbours)
    uint64_t *out[15];
    const uint16_t *elig[15];    // per colour c, the E ranks of the size-h sets holding c
    int E[15];                   // C(k-1, h-1)
    const uint8_t *col;          // colours of the pass, [vertex][colouring]
};
// Lf: limbs of the fused step's sums and rows (Ld or Ld - 1); Ld: the leaf steps'
void launch_gather_select_chain(cudaStream_t st, int Ls, int Lf, int Ld, int64_t v0, int64_t v1, int64_t split,
                                const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int B, int k,
                                int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *add_p,
                                const uint16_t *rm_h, const uint8_t *col, uint64_t *out, int64_t out_vs,
                                const LeafChain &chain, unsigned long long *next, int nb = 4,
                                AbsentSkip sk = {});

// The chain's p = 1 steps for the light vertices of [v0, v1) whose first-step
// rows are at out0 + (v - v0) * out_vs (written by launch_gather_select).
void launch_leaf_chain(cudaStream_t st, int Ld, int64_t v0, int64_t v1, int64_t split, const int64_t *row_ptr, int B,
                       int k, const uint64_t *out0, int64_t out_vs, int64_t Chs, const LeafChain &chain,
                       unsigned long long *next);

// a = 1 combine for heavy vertices [h0, h1) of the heavy list (aggregates from the task path)
void launch_select_heavy(cudaStream_t st, int L, int64_t h0, int64_t h1, int64_t v0, const int32_t *heavy_v, int B,
                         int k, int64_t Ch, int64_t Chs, int64_t Cps, const uint16_t *rm, const uint8_t *col,
                         const uint64_t *agg, uint64_t *out);

// totals[b] += sum_v root[v][b]  (root rows hold C(k,k) = 1 column)
void launch_root_reduce(cudaStream_t st, int L, int64_t nv, int B, const uint64_t *root,
                        uint64_t *scratch, int64_t scratch_ctas, uint64_t *totals);
// graph batches: per member graph totals over the compact vertices [v0, v1)
void launch_member_reduce(cudaStream_t st, int L, int64_t v0, int64_t v1, int B, const uint64_t *root,
                          const int64_t *member_act, int n_members, uint64_t *totals);

// samples: out[(b * n_s + i) * L] = root[sample_local[i]][b] for samples inside [v0, v1)
void launch_sample_extract(cudaStream_t st, int L, int64_t n_s, const int64_t *sample_v,
                           int64_t v0, int64_t v1, int B, const uint64_t *root, uint64_t *out);

// homomorphism bound: H[v] *= sum_{u in N(v)} Hc[u]  (Hc == nullptr: all ones);
// F (if not null) receives the factor sum_{u in N(v)} Hc[u]
void launch_hom_step(cudaStream_t st, int64_t n_act, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *Hc, double *H, double *F = nullptr);
void launch_fill_double(cudaStream_t st, int64_t n, double v, double *x);
// out[0] = max, out[1] = sum (out must be zeroed)
void launch_max_sum(cudaStream_t st, int64_t n, const double *x, double *out);

// relabelled CSR: list of new vertex nv = list of orig[nv] in the input CSR,
// neighbour ids mapped through new_id
void launch_permute_lists(cudaStream_t st, int64_t n_act, int64_t n, const int64_t *orig, const int64_t *old_rp,
                          const int64_t *new_rp, const int32_t *src, const int32_t *new_id, int32_t *dst);
// col_idx remap for the compact numbering: dst[e] = new_id[src[e]]
void launch_remap(cudaStream_t st, int64_t nnz, int64_t n, const int32_t *src, const int32_t *new_id, int32_t *dst);

int64_t reduce_scratch_ctas();

// Row stride (in values) of a table with C colour-set columns: C rounded up to
// even, so every row and row segment is a whole number of 16-byte units.
inline int64_t col_stride(int64_t C) { return (C + 1) & ~int64_t(1); }

}  // namespace cc
