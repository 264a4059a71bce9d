// kernels.cu -- the colour-coding DP kernels (arXiv 1804.09764, Section 2.1).
//
//   colour        Algorithm 1: a colour in [0, k) for every vertex, per colouring
//   hist          leaf gather: Eq. 1's sum over N(v) when T_i'' is one vertex
//   gather_*      Eq. 1's sum over u in N(v) of the passive table rows
//                 (light vertices: one warp per vertex; heavy vertices: the
//                 neighbour list is cut into tasks of at most s neighbours,
//                 the one-GPU form of Algorithm 4, and the partial rows are
//                 summed by gather_reduce)
//   combine_*     Eq. 1's sum over disjoint colour sets S1 u S2 = S
//   root_reduce   Eq. 3's sum over v
// All arithmetic is on unsigned integers modulo 2^(64 L).
#include "kernels.cuh"
#include "wideint.cuh"

#include <algorithm>

namespace cc {

namespace {

constexpr int kWarps = 8;  // warps per CTA for warp-per-row kernels

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t state)
{
    // SplitMix64 output function (Steele, Lea, Flood 2014) of state + golden gamma
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void colour_kernel(int64_t n_act, int B, int k, const int64_t *__restrict__ orig,
                              const ColourParams *__restrict__ prm, uint8_t *__restrict__ col)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_act * B) return;
    int64_t v = i / B;
    int b = (int)(i - v * B);
    uint64_t h = splitmix64_out(prm->hj[b] + (uint64_t)orig[v]);
    col[i] = (uint8_t)__umul64hi(h, (uint64_t)k);
}

// warp per vertex; per-warp shared counters [B][k]
__global__ void hist_kernel(int64_t v0, int64_t v1, int B, int k, const int64_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col_idx, const uint8_t *__restrict__ col,
                            uint32_t *__restrict__ hist)
{
    extern __shared__ uint32_t cnt_all[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *cnt = cnt_all + warp * B * k;
    const int64_t v = v0 + blockIdx.x * (int64_t)kWarps + warp;
    const bool live = v < v1;
    for (int i = lane; i < B * k; i += 32) cnt[i] = 0;
    __syncwarp();
    if (live) {
        const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t u = col_idx[e];
            const uint8_t *cu = col + u * B;
            for (int b = 0; b < B; b++) atomicAdd(&cnt[b * k + cu[b]], 1u);
        }
    }
    __syncwarp();
    if (live) {
        uint32_t *out = hist + v * (int64_t)B * k;
        for (int i = lane; i < B * k; i += 32) out[i] = cnt[i];
    }
}

// Sum rows X[u] over the neighbour sub-list col_idx[e0, e1) into out_row.
// Lane `lane` owns values base + q*32 + lane, q < VPT; the neighbour ids are
// fetched 32 at a time and broadcast with shuffles; two neighbours are loaded
// before adding so 2*VPT loads are in flight per lane.
template <int Ls, int Ld, int VPT>
__device__ __forceinline__ void gather_row(const int32_t *__restrict__ col_idx, int64_t e0, int64_t e1,
                                           const uint64_t *__restrict__ X, int64_t R,
                                           uint64_t *__restrict__ out_row, int lane)
{
    for (int64_t base = 0; base < R; base += 32 * VPT) {
        Wide<Ld> acc[VPT];
#pragma unroll
        for (int q = 0; q < VPT; q++) wzero(acc[q]);
        for (int64_t e = e0; e < e1; e += 32) {
            const int cnt = (e1 - e < 32) ? (int)(e1 - e) : 32;
            const int32_t myu = lane < cnt ? col_idx[e + lane] : 0;
            int t = 0;
            for (; t + 2 <= cnt; t += 2) {
                const int64_t u0 = __shfl_sync(0xffffffffu, myu, t);
                const int64_t u1 = __shfl_sync(0xffffffffu, myu, t + 1);
                const uint64_t *r0 = X + u0 * R * Ls;
                const uint64_t *r1 = X + u1 * R * Ls;
                Wide<Ld> x0[VPT], x1[VPT];
#pragma unroll
                for (int q = 0; q < VPT; q++) {
                    const int64_t c = base + q * 32 + lane;
                    if (c < R) {
                        x0[q] = wload<Ls, Ld>(r0 + c * Ls);
                        x1[q] = wload<Ls, Ld>(r1 + c * Ls);
                    } else {
                        wzero(x0[q]);
                        wzero(x1[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < VPT; q++) {
                    wadd(acc[q], x0[q]);
                    wadd(acc[q], x1[q]);
                }
            }
            if (t < cnt) {
                const int64_t u0 = __shfl_sync(0xffffffffu, myu, t);
                const uint64_t *r0 = X + u0 * R * Ls;
#pragma unroll
                for (int q = 0; q < VPT; q++) {
                    const int64_t c = base + q * 32 + lane;
                    if (c < R) wadd(acc[q], wload<Ls, Ld>(r0 + c * Ls));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const int64_t c = base + q * 32 + lane;
            if (c < R) wstore(out_row + c * Ld, acc[q]);
        }
    }
}

template <int Ls, int Ld, int VPT>
__global__ void __launch_bounds__(kWarps * 32)
gather_light_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                    const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int64_t R,
                    uint64_t *__restrict__ agg)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t v = v0 + blockIdx.x * (int64_t)kWarps + warp;
    if (v >= v1) return;
    const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
    if (e1 - e0 > split) return;  // heavy vertex: handled by tasks
    gather_row<Ls, Ld, VPT>(col_idx, e0, e1, X, R, agg + (v - v0) * R * Ld, lane);
}

template <int Ls, int Ld, int VPT>
__global__ void __launch_bounds__(kWarps * 32)
gather_tasks_kernel(int64_t t0, int64_t t1, const int32_t *__restrict__ col_idx,
                    const int64_t *__restrict__ task_e, const uint64_t *__restrict__ X, int64_t R,
                    uint64_t *__restrict__ partial)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = t0 + blockIdx.x * (int64_t)kWarps + warp;
    if (t >= t1) return;
    gather_row<Ls, Ld, VPT>(col_idx, task_e[2 * t], task_e[2 * t + 1], X, R, partial + (t - t0) * R * Ld,
                            lane);
}

template <int Ld>
__global__ void __launch_bounds__(kWarps * 32)
gather_reduce_kernel(int64_t h0, int64_t h1, int64_t v0, int64_t t0, const int32_t *__restrict__ heavy_v,
                     const int64_t *__restrict__ heavy_tptr, const uint64_t *__restrict__ partial, int64_t R,
                     uint64_t *__restrict__ agg)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t hi = h0 + blockIdx.x * (int64_t)kWarps + warp;
    if (hi >= h1) return;
    const int64_t v = heavy_v[hi];
    const int64_t a = heavy_tptr[hi] - t0, b = heavy_tptr[hi + 1] - t0;
    uint64_t *out = agg + (v - v0) * R * Ld;
    for (int64_t c = lane; c < R; c += 32) {
        Wide<Ld> acc;
        wzero(acc);
        for (int64_t t = a; t < b; t++) wadd(acc, wload<Ld, Ld>(partial + (t * R + c) * Ld));
        wstore(out + c * Ld, acc);
    }
}

template <int L>
__global__ void combine_generic_kernel(int64_t total, int64_t Ch, int64_t Ca, int64_t Cp, int64_t npairs,
                                       const uint32_t *__restrict__ pairs, const uint64_t *__restrict__ act,
                                       const uint64_t *__restrict__ agg, uint64_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = i / Ch, s = i - vb * Ch;
        const uint64_t *ar = act + vb * Ca * L;
        const uint64_t *pr = agg + vb * Cp * L;
        Wide<L> acc;
        wzero(acc);
        for (int64_t q = 0; q < npairs; q++) {
            const uint32_t pq = __ldg(pairs + q * Ch + s);
            wmac(acc, wload<L, L>(ar + (pq & 0xFFFFu) * L), wload<L, L>(pr + (pq >> 16) * L));
        }
        wstore(out + i * L, acc);
    }
}

template <int L, bool HIST>
__global__ void combine_select_kernel(int64_t total, int64_t v0, int B, int k, int64_t Ch, int64_t Cp,
                                      const uint16_t *__restrict__ rm, const uint8_t *__restrict__ col,
                                      const void *__restrict__ aggp, uint64_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = i / Ch, s = i - vb * Ch;
        const int64_t lv = vb / B;
        const int b = (int)(vb - lv * B);
        const int c = col[(v0 + lv) * B + b];
        const uint32_t r = rm[s * k + c];
        Wide<L> x;
        wzero(x);
        if (r != 0xFFFFu) {
            if constexpr (HIST) {
                x.w[0] = reinterpret_cast<const uint32_t *>(aggp)[vb * k + r];
            } else {
                x = wload<L, L>(reinterpret_cast<const uint64_t *>(aggp) + (vb * Cp + r) * L);
            }
        }
        wstore(out + i * L, x);
    }
}

template <int L>
__global__ void combine_hist_kernel(int64_t total, int k, int64_t Ch, int64_t Ca,
                                    const uint16_t *__restrict__ rm, const uint64_t *__restrict__ act,
                                    const uint32_t *__restrict__ hist, uint64_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = i / Ch, s = i - vb * Ch;
        const uint64_t *ar = act + vb * Ca * L;
        const uint32_t *hr = hist + vb * k;
        Wide<L> acc;
        wzero(acc);
        for (int c = 0; c < k; c++) {
            const uint32_t r = rm[s * k + c];
            if (r == 0xFFFFu) continue;
            const uint32_t hc = hr[c];
            if (hc) wmac_small(acc, wload<L, L>(ar + r * L), hc);
        }
        wstore(out + i * L, acc);
    }
}

template <int L>
__device__ __forceinline__ Wide<L> block_sum(Wide<L> x)
{
    __shared__ uint64_t sh[32][L];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d; d >>= 1) wadd(x, wshfl_down(x, d));
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < L; i++) sh[warp][i] = x.w[i];
    __syncthreads();
    Wide<L> r;
    wzero(r);
    if (warp == 0) {
        if (lane < (int)(blockDim.x >> 5))
#pragma unroll
            for (int i = 0; i < L; i++) r.w[i] = sh[lane][i];
#pragma unroll
        for (int d = 16; d; d >>= 1) wadd(r, wshfl_down(r, d));
    }
    __syncthreads();
    return r;
}

template <int L>
__global__ void root_reduce_kernel(int64_t nv, int B, const uint64_t *__restrict__ root,
                                   uint64_t *__restrict__ scratch)
{
    for (int b = 0; b < B; b++) {
        Wide<L> acc;
        wzero(acc);
        for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
             v += (int64_t)gridDim.x * blockDim.x)
            wadd(acc, wload<L, L>(root + (v * B + b) * L));
        Wide<L> s = block_sum(acc);
        if (threadIdx.x == 0) wstore(scratch + ((int64_t)b * gridDim.x + blockIdx.x) * L, s);
    }
}

template <int L>
__global__ void root_final_kernel(int64_t nctas, int B, const uint64_t *__restrict__ scratch,
                                  uint64_t *__restrict__ totals)
{
    const int b = blockIdx.x;
    Wide<L> acc;
    wzero(acc);
    for (int64_t c = threadIdx.x; c < nctas; c += blockDim.x)
        wadd(acc, wload<L, L>(scratch + ((int64_t)b * nctas + c) * L));
    Wide<L> s = block_sum(acc);
    if (threadIdx.x == 0) {
        Wide<L> t;
#pragma unroll
        for (int i = 0; i < L; i++) t.w[i] = totals[(int64_t)b * L + i];
        wadd(t, s);
        wstore(totals + (int64_t)b * L, t);
    }
}

template <int L>
__global__ void sample_kernel(int64_t n_s, const int64_t *__restrict__ sample_v, int64_t v0, int64_t v1,
                              int B, const uint64_t *__restrict__ root, uint64_t *__restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_s * B) return;
    const int64_t s = i / B;
    const int b = (int)(i - s * B);
    const int64_t v = sample_v[s];
    if (v < v0 || v >= v1) return;
    for (int l = 0; l < L; l++) out[((int64_t)b * n_s + s) * L + l] = root[((v - v0) * B + b) * L + l];
}

__global__ void hom_step_kernel(int64_t n_act, const int64_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col_idx, const double *__restrict__ Hc,
                                double *__restrict__ H)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t v = blockIdx.x * (int64_t)kWarps + warp;
    if (v >= n_act) return;
    double s = 0;
    for (int64_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) s += Hc ? Hc[col_idx[e]] : 1.0;
#pragma unroll
    for (int d = 16; d; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) H[v] *= s;
}

__global__ void fill_double_kernel(int64_t n, double v, double *x)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void max_sum_kernel(int64_t n, const double *__restrict__ x, double *out)
{
    double mx = 0, sm = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        mx = fmax(mx, x[i]);
        sm += x[i];
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, d));
        sm += __shfl_down_sync(0xffffffffu, sm, d);
    }
    if ((threadIdx.x & 31) == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long *>(out), (unsigned long long)__double_as_longlong(mx));
        atomicAdd(out + 1, sm);
    }
}

__global__ void remap_kernel(int64_t nnz, const int32_t *__restrict__ src, const int32_t *__restrict__ new_id,
                             int32_t *__restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nnz) dst[i] = new_id[src[i]];
}

inline unsigned grid_for(int64_t items, int per_cta) { return (unsigned)((items + per_cta - 1) / per_cta); }

inline unsigned grid_stride_ctas(int64_t items, int threads)
{
    int64_t g = (items + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <int Ls, int Ld>
void gather_light_t(cudaStream_t st, int64_t v0, int64_t v1, int64_t split, const int64_t *rp,
                    const int32_t *ci, const uint64_t *X, int64_t R, uint64_t *agg)
{
    constexpr int VPT = Ld <= 2 ? 4 : 2;
    gather_light_kernel<Ls, Ld, VPT><<<grid_for(v1 - v0, kWarps), kWarps * 32, 0, st>>>(v0, v1, split, rp, ci,
                                                                                         X, R, agg);
}

template <int Ls, int Ld>
void gather_tasks_t(cudaStream_t st, int64_t t0, int64_t t1, const int32_t *ci, const int64_t *te,
                    const uint64_t *X, int64_t R, uint64_t *partial)
{
    constexpr int VPT = Ld <= 2 ? 4 : 2;
    gather_tasks_kernel<Ls, Ld, VPT><<<grid_for(t1 - t0, kWarps), kWarps * 32, 0, st>>>(t0, t1, ci, te, X, R,
                                                                                         partial);
}

#define CC_DISPATCH_L(L, ...)                  \
    switch (L) {                               \
    case 1: { constexpr int LL = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int LL = 3; __VA_ARGS__; } break; \
    default: { constexpr int LL = 4; __VA_ARGS__; } break; \
    }

}  // namespace

void launch_colour(cudaStream_t st, int64_t n_act, int B, int k, const int64_t *orig_id,
                   const ColourParams *prm, uint8_t *col)
{
    if (n_act == 0) return;
    colour_kernel<<<grid_for(n_act * B, 256), 256, 0, st>>>(n_act, B, k, orig_id, prm, col);
}

void launch_hist(cudaStream_t st, int64_t v0, int64_t v1, int B, int k, const int64_t *row_ptr,
                 const int32_t *col_idx, const uint8_t *col, uint32_t *hist)
{
    if (v1 <= v0) return;
    size_t sh = (size_t)kWarps * B * k * sizeof(uint32_t);
    hist_kernel<<<grid_for(v1 - v0, kWarps), kWarps * 32, sh, st>>>(v0, v1, B, k, row_ptr, col_idx, col, hist);
}

void launch_gather_light(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                         const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int64_t R,
                         uint64_t *agg)
{
    if (v1 <= v0) return;
#define CC_GL(a, b) if (Ls == a && Ld == b) return gather_light_t<a, b>(st, v0, v1, split, row_ptr, col_idx, X, R, agg)
    CC_GL(1, 1); CC_GL(1, 2); CC_GL(1, 3); CC_GL(1, 4);
    CC_GL(2, 1); CC_GL(2, 2); CC_GL(2, 3); CC_GL(2, 4);
    CC_GL(3, 1); CC_GL(3, 2); CC_GL(3, 3); CC_GL(3, 4);
    CC_GL(4, 1); CC_GL(4, 2); CC_GL(4, 3); CC_GL(4, 4);
#undef CC_GL
}

void launch_gather_tasks(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                         const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial)
{
    if (t1 <= t0) return;
#define CC_GT(a, b) if (Ls == a && Ld == b) return gather_tasks_t<a, b>(st, t0, t1, col_idx, task_e, X, R, partial)
    CC_GT(1, 1); CC_GT(1, 2); CC_GT(1, 3); CC_GT(1, 4);
    CC_GT(2, 1); CC_GT(2, 2); CC_GT(2, 3); CC_GT(2, 4);
    CC_GT(3, 1); CC_GT(3, 2); CC_GT(3, 3); CC_GT(3, 4);
    CC_GT(4, 1); CC_GT(4, 2); CC_GT(4, 3); CC_GT(4, 4);
#undef CC_GT
}

void launch_gather_reduce(cudaStream_t st, int Ld, int64_t h0, int64_t h1, int64_t v0, int64_t t0,
                          const int32_t *heavy_v, const int64_t *heavy_tptr, const uint64_t *partial, int64_t R,
                          uint64_t *agg)
{
    if (h1 <= h0) return;
    CC_DISPATCH_L(Ld, gather_reduce_kernel<LL><<<grid_for(h1 - h0, kWarps), kWarps * 32, 0, st>>>(
                          h0, h1, v0, t0, heavy_v, heavy_tptr, partial, R, agg));
}

void launch_combine_generic(cudaStream_t st, int L, int64_t nv, int B, int64_t Ch, int64_t Ca, int64_t Cp,
                            int64_t npairs, const uint32_t *pairs, const uint64_t *act, const uint64_t *agg,
                            uint64_t *out)
{
    const int64_t total = nv * B * Ch;
    if (total == 0) return;
    CC_DISPATCH_L(L, combine_generic_kernel<LL><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                         total, Ch, Ca, Cp, npairs, pairs, act, agg, out));
}

void launch_combine_select(cudaStream_t st, int L, bool agg_is_hist, int64_t v0, int64_t nv, int B, int k,
                           int64_t Ch, int64_t Cp, const uint16_t *rm, const uint8_t *col, const void *agg,
                           uint64_t *out)
{
    const int64_t total = nv * B * Ch;
    if (total == 0) return;
    if (agg_is_hist) {
        CC_DISPATCH_L(L, combine_select_kernel<LL, true><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                             total, v0, B, k, Ch, Cp, rm, col, agg, out));
    } else {
        CC_DISPATCH_L(L, combine_select_kernel<LL, false><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                             total, v0, B, k, Ch, Cp, rm, col, agg, out));
    }
}

void launch_combine_hist(cudaStream_t st, int L, int64_t v0, int64_t nv, int B, int k, int64_t Ch, int64_t Ca,
                         int h, const uint16_t *rm, const uint64_t *act, const uint32_t *hist, uint64_t *out)
{
    (void)v0;
    (void)h;
    const int64_t total = nv * B * Ch;
    if (total == 0) return;
    CC_DISPATCH_L(L, combine_hist_kernel<LL><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                         total, k, Ch, Ca, rm, act, hist, out));
}

int64_t reduce_scratch_ctas() { return 152 * 2; }

void launch_root_reduce(cudaStream_t st, int L, int64_t nv, int B, const uint64_t *root, uint64_t *scratch,
                        int64_t scratch_ctas, uint64_t *totals)
{
    if (nv == 0) return;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(scratch_ctas, (nv + 255) / 256));
    CC_DISPATCH_L(L, root_reduce_kernel<LL><<<g, 256, 0, st>>>(nv, B, root, scratch));
    CC_DISPATCH_L(L, root_final_kernel<LL><<<B, 256, 0, st>>>(g, B, scratch, totals));
}

void launch_sample_extract(cudaStream_t st, int L, int64_t n_s, const int64_t *sample_v, int64_t v0, int64_t v1,
                           int B, const uint64_t *root, uint64_t *out)
{
    if (n_s == 0) return;
    CC_DISPATCH_L(L, sample_kernel<LL><<<grid_for(n_s * B, 256), 256, 0, st>>>(n_s, sample_v, v0, v1, B, root,
                                                                                out));
}

void launch_hom_step(cudaStream_t st, int64_t n_act, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *Hc, double *H)
{
    if (n_act == 0) return;
    hom_step_kernel<<<grid_for(n_act, kWarps), kWarps * 32, 0, st>>>(n_act, row_ptr, col_idx, Hc, H);
}

void launch_fill_double(cudaStream_t st, int64_t n, double v, double *x)
{
    if (n == 0) return;
    fill_double_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, v, x);
}

void launch_max_sum(cudaStream_t st, int64_t n, const double *x, double *out)
{
    if (n == 0) return;
    max_sum_kernel<<<grid_stride_ctas(n, 256), 256, 0, st>>>(n, x, out);
}

void launch_remap(cudaStream_t st, int64_t nnz, const int32_t *src, const int32_t *new_id, int32_t *dst)
{
    if (nnz == 0) return;
    remap_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, src, new_id, dst);
}

}  // namespace cc
