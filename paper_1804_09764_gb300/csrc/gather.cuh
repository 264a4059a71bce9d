// gather.cuh -- device and launch helpers shared by the gather kernels
// (kernels.cu) and the fused gather + combine kernels (fused.cu).  Internal to
// the library: everything is in an unnamed namespace, one copy per file.
#pragma once

#include "kernels.cuh"
#include "wideint.cuh"

#include <algorithm>
#include <map>
#include <mutex>

namespace cc {

namespace {

constexpr int kWarps = 8;  // warps per CTA for warp-per-row kernels

// Bulk prefetch of a contiguous range into L2 (no registers, no completion
// tracking): the row of a neighbour is requested whole as soon as its id is
// known, so the chunked loads that follow mostly hit L2.  Range and address
// are multiples of 16 bytes (rows have an even number of 8-byte limbs).
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Neighbour ids travel through the warp with the neighbour's colour in bits
// 27..30 when absent entries are skipped (AbsentSkip); kIdBits masks the id.
constexpr uint32_t kIdBits = (1u << 27) - 1;

// Per-lane skip state of one sweep: m[q] = the colour mask of value base +
// q * 32 + lane (all colours without skipping, 0 past the row), idm = the id
// bits of a broadcast neighbour word.
template <int VPT>
struct LaneMask {
    uint32_t m[VPT];
    uint32_t idm;
    __device__ __forceinline__ void init(const AbsentSkip &sk, int64_t R, int64_t base, int lane)
    {
        idm = sk.ncol ? kIdBits : 0x7fffffffu;
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const int64_t c = base + q * 32 + lane;
            m[q] = c < R ? (sk.ncol ? (uint32_t)__ldg(sk.smask + c) : 0xffffu) : 0u;
        }
    }
    // this lane's word for list entry e (lane < cnt): the id, with the colour above it
    __device__ __forceinline__ int32_t word(const AbsentSkip &sk, const int32_t *__restrict__ col_idx, int64_t e) const
    {
        int32_t w = __ldg(col_idx + e);
        if (sk.ncol) w |= (int32_t)((uint32_t)__ldg(sk.ncol + e) << 27);
        return w;
    }
};

// One batch of NB neighbours (words in lanes t .. t + NB - 1 of myu) of the row
// sums below: every load of the batch is issued before any is added, NB * VPT
// loads in flight per lane.  xl points at value base + lane of row 0; row u
// starts rb * u bytes further; a value is loaded only where its colour mask
// holds the neighbour's colour (the others are zero, AbsentSkip).
template <int Ls, int Ld, int VPT, int NB>
__device__ __forceinline__ void sum_batch(RowSum<Ls, Ld> (&s)[VPT], const char *xl, uint32_t rb, int32_t myu, int t,
                                          const LaneMask<VPT> &lm)
{
    using S = RowSum<Ls, Ld>;
    Wide<S::N> x[NB][VPT];
#pragma unroll
    for (int j = 0; j < NB; j++) {
        const uint32_t w = (uint32_t)__shfl_sync(0xffffffffu, myu, t + j);
        const uint32_t bit = 1u << (w >> 27);
        const uint64_t *row = reinterpret_cast<const uint64_t *>(xl + (uint64_t)(w & lm.idm) * rb);
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            if (lm.m[q] & bit)
                x[j][q] = S::load(row + q * 32 * Ls);
            else
                wzero(x[j][q]);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; j++)
#pragma unroll
        for (int q = 0; q < VPT; q++) s[q].add(x[j][q]);
}

// acc[q] = the sum of X[u][base + q*32 + lane] over the neighbours u of
// col_idx[e0, e1) (values of Ls limbs summed to Ld limbs with a carry counter,
// RowSum; entries at or beyond R are left zero).  Neighbour ids are fetched 32
// at a time and broadcast with shuffles; neighbours go NB at a time, the rest
// one by one.  Row addresses are one 32 x 32 -> 64-bit multiply-add per
// neighbour (rows are less than 4 GiB apart), column offsets are constants.
template <int Ls, int Ld, int VPT, int NB>
__device__ __forceinline__ void accumulate_rows_counted(const int32_t *__restrict__ col_idx, int64_t e0,
                                                        int64_t e1, const uint64_t *__restrict__ X, int64_t R,
                                                        int64_t base, Wide<Ld> (&acc)[VPT], int lane,
                                                        const AbsentSkip &sk)
{
    RowSum<Ls, Ld> s[VPT];
    LaneMask<VPT> lm;
    lm.init(sk, R, base, lane);
#pragma unroll
    for (int q = 0; q < VPT; q++) s[q].zero();
    const char *xl = reinterpret_cast<const char *>(X + (base + lane) * Ls);
    const uint32_t rb = (uint32_t)(R * Ls * 8);
    for (int64_t e = e0; e < e1; e += 32) {
        const int cnt = (e1 - e < 32) ? (int)(e1 - e) : 32;
        const int32_t myu = lane < cnt ? lm.word(sk, col_idx, e + lane) : 0;
        const int nfull = cnt - cnt % NB;
        for (int t = 0; t < nfull; t += NB) sum_batch<Ls, Ld, VPT, NB>(s, xl, rb, myu, t, lm);
        for (int t = nfull; t < cnt; t++) sum_batch<Ls, Ld, VPT, 1>(s, xl, rb, myu, t, lm);
    }
#pragma unroll
    for (int q = 0; q < VPT; q++) acc[q] = s[q].wide();
}

// acc[q] += X[u][base + q*32 + lane] over the neighbours u of col_idx[e0, e1)
// with full Ld-limb adds: neighbour ids are fetched 32 at a time and broadcast
// with shuffles, and NB neighbours' values are loaded before any is added
// (NB * VPT loads in flight per lane).  Absent entries are skipped as above.
template <int Ls, int Ld, int VPT, int NB>
__device__ __forceinline__ void accumulate_rows_limbwise(const int32_t *__restrict__ col_idx, int64_t e0,
                                                         int64_t e1, const uint64_t *__restrict__ X, int64_t R,
                                                         int64_t base, Wide<Ld> (&acc)[VPT], int lane,
                                                         const AbsentSkip &sk)
{
    LaneMask<VPT> lm;
    lm.init(sk, R, base, lane);
    for (int64_t e = e0; e < e1; e += 32) {
        const int cnt = (e1 - e < 32) ? (int)(e1 - e) : 32;
        const int32_t myu = lane < cnt ? lm.word(sk, col_idx, e + lane) : 0;
        int t = 0;
        for (; t + NB <= cnt; t += NB) {
            Wide<Ld> x[NB][VPT];
#pragma unroll
            for (int j = 0; j < NB; j++) {
                const uint32_t w = (uint32_t)__shfl_sync(0xffffffffu, myu, t + j);
                const uint32_t bit = 1u << (w >> 27);
                const uint64_t *row = X + (int64_t)(w & lm.idm) * R * Ls;
#pragma unroll
                for (int q = 0; q < VPT; q++) {
                    const int64_t c = base + q * 32 + lane;
                    if (lm.m[q] & bit)
                        x[j][q] = wload<Ls, Ld>(row + c * Ls);
                    else
                        wzero(x[j][q]);
                }
            }
#pragma unroll
            for (int j = 0; j < NB; j++)
#pragma unroll
                for (int q = 0; q < VPT; q++) wadd(acc[q], x[j][q]);
        }
        for (; t < cnt; t++) {
            const uint32_t w = (uint32_t)__shfl_sync(0xffffffffu, myu, t);
            const uint32_t bit = 1u << (w >> 27);
            const uint64_t *row = X + (int64_t)(w & lm.idm) * R * Ls;
#pragma unroll
            for (int q = 0; q < VPT; q++) {
                const int64_t c = base + q * 32 + lane;
                if (lm.m[q] & bit) wadd(acc[q], wload<Ls, Ld>(row + c * Ls));
            }
        }
    }
}

// acc[q] (zero on entry) = the neighbour sum of value base + q * 32 + lane.
// One-limb sources take the carry-counter form (one 64-bit add and a 32-bit
// carry add per value instead of a full two-limb add); wider sources keep the
// limb-wise form, the one measured for the root chain's <2,2,3> instantiation
// without a register cap (17 ms per launch on R-MAT s22 / tree-12, against
// 23 ms under a three-CTA cap with either form).
template <int Ls, int Ld, int VPT, int NB>
__device__ __forceinline__ void accumulate_rows(const int32_t *__restrict__ col_idx, int64_t e0, int64_t e1,
                                                const uint64_t *__restrict__ X, int64_t R, int64_t base,
                                                Wide<Ld> (&acc)[VPT], int lane, const AbsentSkip &sk)
{
    if constexpr (Ls == 1)
        accumulate_rows_counted<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane, sk);
    else
        accumulate_rows_limbwise<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane, sk);
}

// Sum rows X[u] over the neighbour sub-list col_idx[e0, e1) into out_row.
// Lane `lane` owns values base + q*32 + lane, q < VPT; the neighbour ids are
// fetched 32 at a time and broadcast with shuffles; two neighbours are loaded
// before adding so 2*VPT loads are in flight per lane.
template <int Ls, int Ld, int VPT, bool PF = false, int NB = 2>
__device__ __forceinline__ void gather_row(const int32_t *__restrict__ col_idx, int64_t e0, int64_t e1,
                                           const uint64_t *__restrict__ X, int64_t R,
                                           uint64_t *__restrict__ out_row, int lane, const AbsentSkip &sk)
{
    for (int64_t base = 0; base < R; base += 32 * VPT) {
        Wide<Ld> acc[VPT];
#pragma unroll
        for (int q = 0; q < VPT; q++) wzero(acc[q]);
        if (PF && base == 0 && R > 32 * VPT && (R * Ls) % 2 == 0)
            for (int64_t e = e0 + lane; e < e1; e += 32)
                prefetch_l2(X + (int64_t)col_idx[e] * R * Ls, (uint32_t)(R * Ls * 8));
        accumulate_rows<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane, sk);
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const int64_t c = base + q * 32 + lane;
            if (c < R) wstore(out_row + c * Ld, acc[q]);
        }
    }
}

// Values [b0, b1) of the sum of rows X[u] over col_idx[e0, e1) into out_row
// (b0 a multiple of 32 * VPT; b1 <= R).
template <int Ls, int Ld, int VPT, int NB>
__device__ __forceinline__ void gather_row_range(const int32_t *__restrict__ col_idx, int64_t e0, int64_t e1,
                                                 const uint64_t *__restrict__ X, int64_t R, int64_t b0, int64_t b1,
                                                 uint64_t *__restrict__ out_row, int lane, const AbsentSkip &sk)
{
    for (int64_t base = b0; base < b1; base += 32 * VPT) {
        Wide<Ld> acc[VPT];
#pragma unroll
        for (int q = 0; q < VPT; q++) wzero(acc[q]);
        accumulate_rows<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, base, acc, lane, sk);
#pragma unroll
        for (int q = 0; q < VPT; q++) {
            const int64_t c = base + q * 32 + lane;
            if (c < b1) wstore(out_row + c * Ld, acc[q]);
        }
    }
}

// Position (b, s) of the flat index i = b * stride + s in a vertex's rows (B
// colourings of `stride` entries each), moved forward without a division per
// entry: one 32-bit division to start, then steps of the 32 entries a warp
// covers per sweep.  Row sizes stay below 2^31 (B <= 64, stride <= 12870).
struct RowPos {
    int b, s;
    __device__ __forceinline__ void init(int i, int stride)
    {
        b = i / stride;
        s = i - b * stride;
    }
    __device__ __forceinline__ void step(int d, int stride)
    {
        s += d;
        while (s >= stride) {
            s -= stride;
            b++;
        }
    }
};

// Width of one of nch column segments of a row of R values: a multiple of the
// 32 * VPT values a warp covers per sweep.
template <int VPT>
__device__ __forceinline__ int64_t segment_width(int64_t R, int nch)
{
    const int64_t per = (R + nch - 1) / nch;
    return (per + 32 * VPT - 1) / (32 * VPT) * (32 * VPT);
}

inline unsigned grid_for(int64_t items, int per_cta) { return (unsigned)((items + per_cta - 1) / per_cta); }

inline unsigned grid_stride_ctas(int64_t items, int threads)
{
    int64_t g = (items + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// persistent grid size: resident CTAs per SM x SMs (queried once per kernel)
template <typename K>
unsigned persistent_ctas(K kernel)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;  // (kernel, device) -> CTAs
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(reinterpret_cast<const void *>(kernel), dev);
    auto it = cache.find(key);
    if (it != cache.end()) return (unsigned)it->second;
    int per_sm = 1, sms = 152;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarps * 32, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int n = std::max(1, per_sm) * sms;
    cache[key] = n;
    return (unsigned)n;
}

#define CC_DISPATCH_L(L, ...)                  \
    switch (L) {                               \
    case 1: { constexpr int LL = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int LL = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int LL = 3; __VA_ARGS__; } break; \
    default: { constexpr int LL = 4; __VA_ARGS__; } break; \
    }

}  // namespace

}  // namespace cc
