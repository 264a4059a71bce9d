// fused.cu -- Eq. 1 with T_i' a single vertex (a = 1) as one kernel: the
// table gather sum over u in N(v) of X[u] scattered straight into the step's
// output, and the chain's following leaf steps (p = 1) for the same vertex
// (arXiv 1804.09764, Section 2.1).
#include "gather.cuh"

namespace cc {

namespace {

// Fused gather + a = 1 combine (Eq. 1 with T_i' a single vertex): the sum of
// the neighbour rows agg[T] goes straight to out[T u {col(v)}] (skipped when
// col(v) is in T); entries S of the output with col(v) not in S are zero.  The
// aggregate never reaches memory.  Persistent warps pull light vertices from
// `next`; heavy vertices are left to the task path.
template <int Ls, int Ld, int VPT, int NB = 2>
__global__ void __launch_bounds__(kWarps * 32)
gather_select_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                     const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int B, int k,
                     int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *__restrict__ add_p,
                     const uint16_t *__restrict__ rm_h, const uint8_t *__restrict__ col,
                     uint64_t *__restrict__ out, int64_t out_vs, unsigned long long *next, int nch, int G)
{
    const int lane = threadIdx.x & 31;
    const int64_t R = (int64_t)B * Cps;
    const int64_t ngrp = (v1 - v0 + G - 1) / G, cw = segment_width<VPT>(R, nch);
    while (true) {
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(next, 1ull);
        const int64_t i = (int64_t)__shfl_sync(0xffffffffu, got, 0);
        if (i >= ngrp * nch) return;
        const int64_t seg = i / ngrp, grp = i - seg * ngrp;
        const int64_t va = v0 + grp * G, vb = min(v1, va + G);
        for (int64_t v = va; v < vb; v++) {
            const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
            if (e1 - e0 > split) continue;  // heavy vertex: tasks, reduce, select
            uint64_t *orow = out + (v - v0) * out_vs;
            const uint8_t *cv = col + v * B;
            // zeros where the vertex's colour is not in S (and in the padding):
            // written by segment 0 only; no segment scatters to these entries
            if (seg == 0)
                for (int64_t i2 = lane; i2 < (int64_t)B * Chs; i2 += 32) {
                    const int64_t b = i2 / Chs, S = i2 - b * Chs;
                    if (S >= Ch || rm_h[S * k + cv[b]] == 0xFFFFu) {
                        Wide<Ld> z;
                        wzero(z);
                        wstore(orow + i2 * Ld, z);
                    }
                }
            const int64_t b1 = min(R, (seg + 1) * cw);
            for (int64_t base = seg * cw; base < b1; base += 32 * VPT) {
                Wide<Ld> acc[VPT];
#pragma unroll
                for (int q = 0; q < VPT; q++) wzero(acc[q]);
                accumulate_rows<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane);
                // scatter: agg column T of colouring b lands on T u {col}
#pragma unroll
                for (int q = 0; q < VPT; q++) {
                    const int64_t c = base + q * 32 + lane;
                    if (c < b1) {
                        const int64_t b = c / Cps, T = c - b * Cps;
                        if (T < Cp) {
                            const uint32_t d = add_p[T * k + cv[b]];
                            if (d != 0xFFFFu) wstore(orow + (b * Chs + d) * Ld, acc[q]);
                        }
                    }
                }
            }
        }
    }
}

// The chain's p = 1 steps for vertex v, from its first-step row orow (stride
// Chs per colouring, Lf-limb values; Lf <= Ld): out_j[S] = sum over c in S of
// out_{j-1}[S \ {c}] * hist[v][c], written with Ld limbs.  The warp reads in
// step j the rows its lanes wrote in step j - 1 (__syncwarp).
template <int Ld, int Lf = Ld>
__device__ __forceinline__ void leaf_steps(int64_t v, int64_t v0, const uint64_t *orow, int64_t Chs,
                                           const LeafChain &chain, int B, int k, int lane)
{
    const uint64_t *prev = orow;
    int64_t prev_s = Chs;
    for (int j = 0; j < chain.n; j++) {
        __syncwarp();
        const uint32_t *hr = chain.hist[j] + v * (int64_t)B * k;
        const int64_t cj = chain.Ch[j], csj = chain.Chs[j];
        const int hj = chain.h[j];
        const uint32_t *pt = chain.pairs[j];
        uint64_t *dst = chain.out[j] + (v - v0) * chain.vs[j];
        for (int64_t i = lane; i < (int64_t)B * csj; i += 32) {
            const int64_t b = i / csj, S = i - b * csj;
            Wide<Ld> acc;
            wzero(acc);
            if (S < cj) {
                const int Lp = j == 0 ? Lf : Ld;  // limbs of the rows read
                const uint64_t *ar = prev + b * prev_s * Lp;
                const uint32_t *hb = hr + b * k;
                for (int q = 0; q < hj; q++) {
                    const uint32_t pq = __ldg(pt + q * cj + S);
                    const uint32_t hc = hb[pq >> 16];
                    if (hc) {
                        Wide<Ld> a;
#pragma unroll
                        for (int l = 0; l < Ld; l++) a.w[l] = l < Lp ? ar[(pq & 0xFFFFu) * Lp + l] : 0;
                        wmac_small(acc, a, hc);
                    }
                }
            }
            wstore(dst + i * Ld, acc);
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
__global__ void __launch_bounds__(kWarps * 32)
gather_select_chain_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                           const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int B, int k,
                           int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *__restrict__ add_p,
                           const uint16_t *__restrict__ rm_h, const uint8_t *__restrict__ col, uint64_t *out,
                           int64_t out_vs, LeafChain chain, unsigned long long *next)
{
    const int lane = threadIdx.x & 31;
    const int64_t R = (int64_t)B * Cps;
    while (true) {
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(next, 1ull);
        const int64_t v = v0 + (int64_t)__shfl_sync(0xffffffffu, got, 0);
        if (v >= v1) return;
        const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        if (e1 - e0 > split) continue;  // heavy vertex: tasks, reduce, select, p = 1 kernels
        uint64_t *orow = out + (v - v0) * out_vs;
        const uint8_t *cv = col + v * B;
        for (int64_t i = lane; i < (int64_t)B * Chs; i += 32) {
            const int64_t b = i / Chs, S = i - b * Chs;
            if (S >= Ch || rm_h[S * k + cv[b]] == 0xFFFFu) {
                Wide<Lf> z;
                wzero(z);
                wstore(orow + i * Lf, z);
            }
        }
        for (int64_t base = 0; base < R; base += 32 * VPT) {
            Wide<Lf> acc[VPT];
#pragma unroll
            for (int q = 0; q < VPT; q++) wzero(acc[q]);
            accumulate_rows<Ls, Lf, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane);
#pragma unroll
            for (int q = 0; q < VPT; q++) {
                const int64_t c = base + q * 32 + lane;
                if (c < R) {
                    const int64_t b = c / Cps, T = c - b * Cps;
                    if (T < Cp) {
                        const uint32_t d = add_p[T * k + cv[b]];
                        if (d != 0xFFFFu) wstore(orow + (b * Chs + d) * Lf, acc[q]);
                    }
                }
            }
        }
        leaf_steps<Ld, Lf>(v, v0, orow, Chs, chain, B, k, lane);
    }
}

// The chain's p = 1 steps for light vertices whose first-step rows were
// written by a previous kernel (rows of vertex v at out0 + (v - v0) * out_vs).
template <int Ld>
__global__ void __launch_bounds__(kWarps * 32)
leaf_chain_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr, int B, int k,
                  const uint64_t *out0, int64_t out_vs, int64_t Chs, LeafChain chain,
                  unsigned long long *next)
{
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(next, 1ull);
        const int64_t v = v0 + (int64_t)__shfl_sync(0xffffffffu, got, 0);
        if (v >= v1) return;
        if (row_ptr[v + 1] - row_ptr[v] > split) continue;  // heavy: the p = 1 kernels
        leaf_steps<Ld>(v, v0, out0 + (v - v0) * out_vs, Chs, chain, B, k, lane);
    }
}

}  // namespace

namespace {

template <int Ls, int Ld>
void gather_select_t(cudaStream_t st, int nb, int64_t v0, int64_t v1, int64_t split, const int64_t *rp,
                     const int32_t *ci, const uint64_t *X, int B, int k, int64_t Cp, int64_t Cps, int64_t Ch,
                     int64_t Chs, const uint16_t *add_p, const uint16_t *rm_h, const uint8_t *col, uint64_t *out,
                     unsigned long long *next, int nch, int G, int64_t out_vs)
{
    constexpr int VPT = Ld <= 2 ? 4 : 2;
    auto kfn = nb == 4 ? gather_select_kernel<Ls, Ld, VPT, 4> : gather_select_kernel<Ls, Ld, VPT, 2>;
    const int64_t items = (v1 - v0 + G - 1) / G * nch;
    const unsigned g = std::min<unsigned>(persistent_ctas(kfn), grid_for(items, kWarps));
    note_launch("gather_select_kernel", Ls, Ld);
    kfn<<<g, kWarps * 32, 0, st>>>(v0, v1, split, rp, ci, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out,
                                   out_vs > 0 ? out_vs : (int64_t)B * Chs * Ld, next, nch, G);
}

}  // namespace

void launch_gather_select(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                          const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int B, int k,
                          int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *add_p,
                          const uint16_t *rm_h, const uint8_t *col, uint64_t *out, unsigned long long *next, int nb,
                          int nch, int G, int64_t out_vs)
{
    if (v1 <= v0) return;
    nch = std::max(1, std::min(nch, 64));
    G = std::max(1, G);
#define CC_GS(a, b) if (Ls == a && Ld == b) return gather_select_t<a, b>(st, nb, v0, v1, split, row_ptr, col_idx, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out, next, nch, G, out_vs)
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
                           unsigned long long *next)
{
    constexpr int VPT = Lf <= 2 ? 4 : 2;
    auto kfn = nb == 4 ? gather_select_chain_kernel<Ls, Lf, Ld, VPT, 4> : gather_select_chain_kernel<Ls, Lf, Ld, VPT, 2>;
    const unsigned g = std::min<unsigned>(persistent_ctas(kfn), grid_for(v1 - v0, kWarps));
    note_launch("gather_select_chain_kernel", Ls, Lf, Ld);
    kfn<<<g, kWarps * 32, 0, st>>>(v0, v1, split, rp, ci, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out,
                                   out_vs, chain, next);
}

}  // namespace

void launch_gather_select_chain(cudaStream_t st, int Ls, int Lf, int Ld, int64_t v0, int64_t v1, int64_t split,
                                const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int B, int k,
                                int64_t Cp, int64_t Cps, int64_t Ch, int64_t Chs, const uint16_t *add_p,
                                const uint16_t *rm_h, const uint8_t *col, uint64_t *out, int64_t out_vs,
                                const LeafChain &chain, unsigned long long *next, int nb)
{
    if (v1 <= v0) return;
    // Lf is Ld or Ld - 1 (the fused step's own width, at most one limb narrower)
    if (Lf < Ld - 1 || Lf > Ld || Lf < 1) Lf = Ld;
#define CC_GC(a, f, b) if (Ls == a && Lf == f && Ld == b) return gather_select_chain_t<a, f, b>(st, nb, v0, v1, split, row_ptr, col_idx, X, B, k, Cp, Cps, Ch, Chs, add_p, rm_h, col, out, out_vs, chain, next)
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
