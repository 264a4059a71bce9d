// fused.cu -- Eq. 1 with T_i' a single vertex (a = 1) as one kernel: the
// table gather sum over u in N(v) of X[u] scattered straight into the step's
// output, and the chain's following leaf steps (p = 1) for the same vertex
// (arXiv 1804.09764, Section 2.1).
#include "gather.cuh"

namespace cc {

namespace {

// Zeros of a fused step's output row where the vertex's colour is not in S
// (and in the padding columns): no neighbour sum scatters to these entries.
template <int L>
__device__ __forceinline__ void zero_missing(uint64_t *orow, int B, int k, int Ch, int Chs,
                                             const uint16_t *__restrict__ rm_h, const uint8_t *cv, int lane)
{
    RowPos pos;
    pos.init(lane, Chs);
    for (int i = lane; i < B * Chs; i += 32, pos.step(32, Chs))
        if (pos.s >= Ch || rm_h[pos.s * k + cv[pos.b]] == 0xFFFFu) {
            Wide<L> z;
            wzero(z);
            wstore(orow + (int64_t)i * L, z);
        }
}

// One warp sweep of a fused step: the neighbour sums acc[q] of the values
// base + q * 32 + lane (< b1) of colouring b, set T, go to out[b][T u {col_b}]
// (skipped when col_b is in T).  pos tracks (b, T) of base + lane and is left
// at base + 32 * VPT + lane.
template <int L, int VPT>
__device__ __forceinline__ void scatter_sums(uint64_t *orow, const Wide<L> (&acc)[VPT], int base, int b1, int Cp,
                                             int Cps, int Chs, int k, const uint16_t *__restrict__ add_p,
                                             const uint8_t *cv, RowPos &pos, int lane)
{
#pragma unroll
    for (int q = 0; q < VPT; q++) {
        if (base + q * 32 + lane < b1 && pos.s < Cp) {
            const uint32_t d = add_p[pos.s * k + cv[pos.b]];
            if (d != 0xFFFFu) wstore(orow + ((int64_t)pos.b * Chs + d) * L, acc[q]);
        }
        pos.step(32, Cps);
    }
}

// Resident CTAs per SM the fused kernels are compiled for (the register cap
// follows; 0: the compiler's choice).  Measured on R-MAT s22 / tree-12 (ms
// per launch): one-limb sources summed to two limbs 29 -> 23 at three CTAs
// (80 registers) rather than four (64), the plain fused step 21 -> 15; the
// root chain (two-limb sources) 17 uncapped (76 registers) but 23 capped at
// three CTAs (80); the <1,1,1> chain 5.5 uncapped (60) against 6.3 at three.
constexpr int select_ctas_per_sm(int Ls, int Ld) { return Ls == 1 ? 3 : 0; }
constexpr int chain_ctas_per_sm(int Ls, int Lf) { return Ls == 1 && Lf == 2 ? 3 : 0; }

// Fused gather + a = 1 combine (Eq. 1 with T_i' a single vertex): the sum of
// the neighbour rows agg[T] goes straight to out[T u {col(v)}] (skipped when
// col(v) is in T); entries S of the output with col(v) not in S are zero.  The
// aggregate never reaches memory.  Persistent warps pull work items from
// `next` (the next claim is requested while the current item runs); heavy
// vertices are left to the task path.
template <int Ls, int Ld, int VPT, int NB = 2>
__global__ void __launch_bounds__(kWarps * 32, select_ctas_per_sm(Ls, Ld))
gather_select_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                     const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int B, int k,
                     int Cp, int Cps, int Ch, int Chs, const uint16_t *__restrict__ add_p,
                     const uint16_t *__restrict__ rm_h, const uint8_t *__restrict__ col,
                     uint64_t *__restrict__ out, int64_t out_vs, unsigned long long *next, int nch, int G,
                     AbsentSkip sk)
{
    const int lane = threadIdx.x & 31;
    const int R = B * Cps;
    const int64_t ngrp = (v1 - v0 + G - 1) / G;
    const int cw = (int)segment_width<VPT>(R, nch);
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(next, 1ull);
    int64_t i = (int64_t)__shfl_sync(0xffffffffu, got, 0);
    while (i < ngrp * nch) {
        if (lane == 0) got = atomicAdd(next, 1ull);  // the next item, awaited after this one
        const int64_t seg = i / ngrp, grp = i - seg * ngrp;
        const int64_t va = v0 + grp * G, vb = min(v1, va + G);
        for (int64_t v = va; v < vb; v++) {
            const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
            if (e1 - e0 > split) continue;  // heavy vertex: tasks, reduce, select
            uint64_t *orow = out + (v - v0) * out_vs;
            const uint8_t *cv = col + v * B;
            if (seg == 0) zero_missing<Ld>(orow, B, k, Ch, Chs, rm_h, cv, lane);  // no segment scatters there
            const int b0 = (int)seg * cw, b1 = min(R, b0 + cw);
            RowPos pos;
            pos.init(b0 + lane, Cps);
            for (int base = b0; base < b1; base += 32 * VPT) {
                Wide<Ld> acc[VPT];
#pragma unroll
                for (int q = 0; q < VPT; q++) wzero(acc[q]);
                accumulate_rows<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane, sk);
                scatter_sums<Ld, VPT>(orow, acc, base, b1, Cp, Cps, Chs, k, add_p, cv, pos, lane);
            }
        }
        i = (int64_t)__shfl_sync(0xffffffffu, got, 0);
    }
}

// The chain's p = 1 steps for vertex v, from its first-step row orow (stride
// Chs per colouring, Lf-limb values; Lf <= Ld): out_j[S] = sum over c in S of
// out_{j-1}[S \ {c}] * hist[v][c], written with Ld limbs.  The warp reads in
// step j the rows its lanes wrote in step j - 1 (__syncwarp).
// Every row of the chain is zero at the sets without v's own colour col(v)
// (the rooted subtree contains v), so a step computes only the C(k-1, h-1)
// outputs S holding col(v) (chain.elig), and of their terms only those with
// c != col(v) (prev[S \ {col(v)}] lacks col(v)); the sets a step reads are
// therefore all ones holding col(v), and only the chain's table (the last
// step, read in full by later gathers) gets its zeros written.  Only the
// colours that some neighbour of v has (in any colouring of the pass) give
// non-zero terms: when they are fewer than half of |S| the sum runs over them
// (rm_h[S * k + c]: rank of S \ {c}, or c outside S), otherwise over the
// split table of S, QB terms loaded at a time (fewer for wide values, to stay
// within the registers of three CTAs per SM).
template <int Ld, int Lf = Ld, int QB = (Ld >= 3 ? 2 : 4)>
__device__ __forceinline__ void leaf_steps(int64_t v, int64_t v0, const uint64_t *orow, int Chs,
                                           const LeafChain &chain, int B, int k, int lane)
{
    const uint64_t *prev = orow;
    int prev_s = Chs;
    const int Bk = B * k;
    const uint8_t *cv = chain.col + v * B;
    for (int j = 0; j < chain.n; j++) {
        const uint32_t *hr = chain.hist[j] + v * (int64_t)Bk;
        // neighbour colour counts; with B * k <= 32 they stay in the lanes'
        // registers and are read with shuffles
        const uint32_t hv = lane < Bk ? hr[lane] : 0u;
        unsigned nz = 0;
        for (int t = lane; t < Bk; t += 32)
            if ((t < 32 ? hv : hr[t]) != 0) nz |= 1u << (t % k);
        nz = __reduce_or_sync(0xffffffffu, nz);
        __syncwarp();
        const int cj = (int)chain.Ch[j], csj = (int)chain.Chs[j], hj = chain.h[j], E = chain.E[j];
        const bool sparse = 2 * __popc(nz) < hj;
        const uint16_t *__restrict__ rm = chain.rm[j];
        const uint16_t *__restrict__ el = chain.elig[j];
        const uint32_t *__restrict__ pt = chain.pairs[j];
        uint64_t *dst = chain.out[j] + (v - v0) * chain.vs[j];
        const int Lp = j == 0 ? Lf : Ld;  // limbs of the rows read
        if (j + 1 == chain.n) {
            // the chain's table: zeros at the sets without col(v) and in the padding
            RowPos zp;
            zp.init(lane, csj);
            for (int i = lane; i < B * csj; i += 32, zp.step(32, csj))
                if (zp.s >= cj || rm[zp.s * k + cv[zp.b]] == 0xFFFFu) {
                    Wide<Ld> z;
                    wzero(z);
                    wstore(dst + (int64_t)i * Ld, z);
                }
        }
        // count of colour c among the neighbours, colouring b (all lanes call it)
        auto count_of = [&](int b, int c, bool live) -> uint32_t {
            if (Bk <= 32) return __shfl_sync(0xffffffffu, hv, (b * k + c) & 31);
            return live ? hr[b * k + c] : 0u;
        };
        RowPos pos;  // (colouring, index among the E sets holding its col(v))
        pos.init(lane, E);
        for (int i0 = 0; i0 < B * E; i0 += 32, pos.step(32, E)) {
            const bool live = i0 + lane < B * E;
            const int cb = live ? cv[pos.b] : 0;  // col(v) in this lane's colouring
            const int S = live ? el[cb * E + pos.s] : 0;
            const uint64_t *ar = prev + (int64_t)pos.b * prev_s * Lp;
            Wide<Ld> acc;
            wzero(acc);
            if (sparse) {
                for (unsigned m = nz; m; m &= m - 1) {
                    const int c = __ffs(m) - 1;
                    const uint32_t hc = count_of(pos.b, c, live);
                    const uint32_t r = live && c != cb ? rm[S * k + c] : 0xFFFFu;
                    if (r != 0xFFFFu && hc) {
                        Wide<Ld> a;
#pragma unroll
                        for (int l = 0; l < Ld; l++) a.w[l] = l < Lp ? ar[(int64_t)r * Lp + l] : 0;
                        wmac_small(acc, a, hc);
                    }
                }
            } else {
                for (int q0 = 0; q0 < hj; q0 += QB) {
                    uint32_t pq[QB], hc[QB];
#pragma unroll
                    for (int t = 0; t < QB; t++) pq[t] = live && q0 + t < hj ? __ldg(pt + (q0 + t) * cj + S) : 0u;
#pragma unroll
                    for (int t = 0; t < QB; t++) {
                        hc[t] = count_of(pos.b, (int)(pq[t] >> 16), live);
                        if (!(live && q0 + t < hj) || (int)(pq[t] >> 16) == cb) hc[t] = 0;
                    }
                    Wide<Ld> a[QB];
#pragma unroll
                    for (int t = 0; t < QB; t++)
#pragma unroll
                        for (int l = 0; l < Ld; l++)
                            a[t].w[l] = (hc[t] && l < Lp) ? ar[(int64_t)(pq[t] & 0xFFFFu) * Lp + l] : 0;
#pragma unroll
                    for (int t = 0; t < QB; t++)
                        if (hc[t]) wmac_small(acc, a[t], hc[t]);
                }
            }
            if (live) wstore(dst + ((int64_t)pos.b * csj + S) * Ld, acc);
        }
        prev = dst;
        prev_s = csj;
    }
}

// Fused gather + a = 1 combine followed, in the same warp, by the chain's p = 1
// steps for that vertex (see LeafChain).  The rows a warp writes are the rows
// it reads next; __syncwarp orders them within the warp.  The fused step sums
// and stores Lf-limb values (the width its own bound needs), the leaf steps Ld.
template <int Ls, int Lf, int Ld, int VPT, int NB>
__global__ void __launch_bounds__(kWarps * 32, chain_ctas_per_sm(Ls, Lf))
gather_select_chain_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int B, int k,
                           int Cp, int Cps, int Ch, int Chs, const uint16_t *__restrict__ add_p,
                           const uint16_t *__restrict__ rm_h, const uint8_t *__restrict__ col, uint64_t *out,
                           int64_t out_vs, LeafChain chain, unsigned long long *next, AbsentSkip sk)
{
    const int lane = threadIdx.x & 31;
    const int R = B * Cps;
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(next, 1ull);
    int64_t v = v0 + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    while (v < v1) {
        if (lane == 0) got = atomicAdd(next, 1ull);  // the next vertex, awaited after this one
        const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        if (e1 - e0 <= split) {  // heavy vertices: tasks, reduce, select, p = 1 kernels
            uint64_t *orow = out + (v - v0) * out_vs;
            const uint8_t *cv = col + v * B;
            // (no zeros: the leaf steps read this row only at sets holding col(v))
            RowPos pos;
            pos.init(lane, Cps);
            for (int base = 0; base < R; base += 32 * VPT) {
                Wide<Lf> acc[VPT];
#pragma unroll
                for (int q = 0; q < VPT; q++) wzero(acc[q]);
                accumulate_rows<Ls, Lf, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane, sk);
                scatter_sums<Lf, VPT>(orow, acc, base, R, Cp, Cps, Chs, k, add_p, cv, pos, lane);
            }
            leaf_steps<Ld, Lf>(v, v0, orow, Chs, chain, B, k, lane);
        }
        v = v0 + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    }
}

// The chain's p = 1 steps for light vertices whose first-step rows were
// written by a previous kernel (rows of vertex v at out0 + (v - v0) * out_vs).
template <int Ld>
__global__ void __launch_bounds__(kWarps * 32)
leaf_chain_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr, int B, int k,
                  const uint64_t *out0, int64_t out_vs, int Chs, LeafChain chain, unsigned long long *next)
{
    const int lane = threadIdx.x & 31;
    unsigned long long got = 0;
    if (lane == 0) got = atomicAdd(next, 1ull);
    int64_t v = v0 + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    while (v < v1) {
        if (lane == 0) got = atomicAdd(next, 1ull);
        if (row_ptr[v + 1] - row_ptr[v] <= split)  // heavy: the p = 1 kernels
            leaf_steps<Ld>(v, v0, out0 + (v - v0) * out_vs, Chs, chain, B, k, lane);
        v = v0 + (int64_t)__shfl_sync(0xffffffffu, got, 0);
    }
}

}  // namespace

namespace {

template <int Ls, int Ld>
void gather_select_t(cudaStream_t st, int nb, int64_t v0, int64_t v1, int64_t split, const int64_t *rp,
                     const int32_t *ci, const uint64_t *X, int B, int k, int64_t Cp, int64_t Cps, int64_t Ch,
                     int64_t Chs, const uint16_t *add_p, const uint16_t *rm_h, const uint8_t *col, uint64_t *out,
                     unsigned long long *next, int nch, int G, int64_t out_vs, AbsentSkip sk)
{
    constexpr int VPT = Ld <= 2 ? 4 : 2;
    auto kfn = nb == 4 ? gather_select_kernel<Ls, Ld, VPT, 4> : gather_select_kernel<Ls, Ld, VPT, 2>;
    const int64_t items = (v1 - v0 + G - 1) / G * nch;
    const unsigned g = std::min<unsigned>(persistent_ctas(kfn), grid_for(items, kWarps));
    note_launch("gather_select_kernel", Ls, Ld);
    kfn<<<g, kWarps * 32, 0, st>>>(v0, v1, split, rp, ci, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out,
                                   out_vs > 0 ? out_vs : (int64_t)B * Chs * Ld, next, nch, G, sk);
}

}  // namespace

void launch_gather_select(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                          const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int B, int k,
                          int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *add_p,
                          const uint16_t *rm_h, const uint8_t *col, uint64_t *out, unsigned long long *next, int nb,
                          int nch, int G, int64_t out_vs, AbsentSkip sk)
{
    if (v1 <= v0) return;
    nch = std::max(1, std::min(nch, 64));
    G = std::max(1, G);
#define CC_GS(a, b) if (Ls == a && Ld == b) return gather_select_t<a, b>(st, nb, v0, v1, split, row_ptr, col_idx, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out, next, nch, G, out_vs, sk)
    CC_GS(1, 1); CC_GS(1, 2); CC_GS(1, 3); CC_GS(1, 4);
    CC_GS(2, 1); CC_GS(2, 2); CC_GS(2, 3); CC_GS(2, 4);
    CC_GS(3, 1); CC_GS(3, 2); CC_GS(3, 3); CC_GS(3, 4);
    CC_GS(4, 1); CC_GS(4, 2); CC_GS(4, 3); CC_GS(4, 4);
#undef CC_GS
}

namespace {

template <int Ls, int Lf, int Ld>
void gather_select_chain_t(cudaStream_t st, int nb, int64_t v0, int64_t v1, int64_t split, const int64_t *rp,
                           const int32_t *ci, const uint64_t *X, int B, int k, int64_t Cp, int64_t Cps, int64_t Ch,
                           int64_t Chs, const uint16_t *add_p, const uint16_t *rm_h, const uint8_t *col,
                           uint64_t *out, int64_t out_vs, const LeafChain &chain,
                           unsigned long long *next, AbsentSkip sk)
{
    constexpr int VPT = Lf <= 2 ? 4 : 2;
    auto kfn = nb == 4 ? gather_select_chain_kernel<Ls, Lf, Ld, VPT, 4> : gather_select_chain_kernel<Ls, Lf, Ld, VPT, 2>;
    const unsigned g = std::min<unsigned>(persistent_ctas(kfn), grid_for(v1 - v0, kWarps));
    note_launch("gather_select_chain_kernel", Ls, Lf, Ld);
    kfn<<<g, kWarps * 32, 0, st>>>(v0, v1, split, rp, ci, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out,
                                   out_vs, chain, next, sk);
}

}  // namespace

void launch_gather_select_chain(cudaStream_t st, int Ls, int Lf, int Ld, int64_t v0, int64_t v1, int64_t split,
                                const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int B, int k,
                                int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *add_p,
                                const uint16_t *rm_h, const uint8_t *col, uint64_t *out, int64_t out_vs,
                                const LeafChain &chain, unsigned long long *next, int nb, AbsentSkip sk)
{
    if (v1 <= v0) return;
    // Lf is Ld or Ld - 1 (the fused step's own width, at most one limb narrower)
    if (Lf < Ld - 1 || Lf > Ld || Lf < 1) Lf = Ld;
#define CC_GC(a, f, b) if (Ls == a && Lf == f && Ld == b) return gather_select_chain_t<a, f, b>(st, nb, v0, v1, split, row_ptr, col_idx, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out, out_vs, chain, next, sk)
#define CC_GC_LS(a) CC_GC(a, 1, 1); CC_GC(a, 1, 2); CC_GC(a, 2, 2); CC_GC(a, 2, 3); CC_GC(a, 3, 3); CC_GC(a, 3, 4); CC_GC(a, 4, 4)
    CC_GC_LS(1); CC_GC_LS(2); CC_GC_LS(3); CC_GC_LS(4);
#undef CC_GC_LS
#undef CC_GC
}

void launch_leaf_chain(cudaStream_t st, int Ld, int64_t v0, int64_t v1, int64_t split, const int64_t *row_ptr, int B,
                       int k, const uint64_t *out0, int64_t out_vs, int64_t Chs, const LeafChain &chain,
                       unsigned long long *next)
{
    if (v1 <= v0 || chain.n <= 0) return;
    CC_DISPATCH_L(Ld, {
        auto kfn = leaf_chain_kernel<LL>;
        const unsigned g = std::min<unsigned>(persistent_ctas(kfn), grid_for(v1 - v0, kWarps));
        note_launch("leaf_chain_kernel", LL);
        kfn<<<g, kWarps * 32, 0, st>>>(v0, v1, split, row_ptr, B, k, out0, out_vs, Chs, chain, next);
    });
}

}  // namespace cc
