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
#include "gather.cuh"

namespace cc {

namespace {

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
                            const uint8_t *__restrict__ labels, int want, uint32_t *__restrict__ hist)
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
            if (labels && labels[u] != want) continue;  // a labelled leaf counts its label only
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

// ---------------------------------------------------------------- bulk-copy gather
//
// Persistent CTAs (one per SM) move whole neighbour-row segments into shared
// memory with cp.async.bulk (TMA), completion tracked by mbarriers, so a few
// hundred KB per SM are in flight with almost no registers.  Warp kBulkConsumers
// (one elected lane) produces: for each work item (a light vertex, or a task of
// a split neighbour list) and each column chunk it walks the neighbour list and
// issues one bulk copy per neighbour into a ring of NS slots.  The consumer
// warps add each staged segment into register accumulators (thread t owns values
// t + q * 256 of the chunk) and free the slot; after the item's last neighbour
// they store the summed chunk.  Every wait is bounded: on timeout the kernel
// records an error code, stops issuing, waits (bounded) for the copies it has
// in flight and returns.
constexpr int kBulkConsumers = 16;                // consumer warps
constexpr int kBulkThreads = (kBulkConsumers + 1) * 32;
constexpr int kBulkMaxStages = 96;
constexpr int64_t kBulkSmemBytes = 192 * 1024;    // stage ring
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false (and *err set) if the phase did not complete in time
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicCAS(err, 0, code);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

struct BulkItems {
    // mode 0: light vertices [v0, v1) with deg <= split, out row = v - v0
    // mode 1: tasks [t0, t1) with ranges task_e, out row = t - t0
    int mode;
    int64_t v0, v1, split;
    const int64_t *row_ptr;
    int64_t t0, t1;
    const int64_t *task_e;
    int64_t nnz;  // length of col_idx
};

// this CTA's item range: vertex ranges balanced by neighbour count, task ranges by count
__device__ __forceinline__ void bulk_item_range(const BulkItems &it, int64_t *a, int64_t *b)
{
    const int64_t G = gridDim.x, g = blockIdx.x;
    if (it.mode == 1) {
        const int64_t n = it.t1 - it.t0, per = (n + G - 1) / G;
        *a = it.t0 + min(n, g * per);
        *b = it.t0 + min(n, (g + 1) * per);
        return;
    }
    const int64_t E0 = it.row_ptr[it.v0], E1 = it.row_ptr[it.v1], E = E1 - E0;
    auto first_at = [&](int64_t target) {  // first v in [v0, v1] with row_ptr[v] >= target
        int64_t lo = it.v0, hi = it.v1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (it.row_ptr[mid] < target) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    *a = (g == 0) ? it.v0 : first_at(E0 + (E * g) / G);
    *b = (g == G - 1) ? it.v1 : first_at(E0 + (E * (g + 1)) / G);
}

// neighbour range of item i (one coalesced load per lane for 32 items at once)
__device__ __forceinline__ void bulk_item_load(const BulkItems &it, int64_t i, int64_t *e0, int64_t *e1)
{
    if (it.mode == 1) {
        *e0 = it.task_e[2 * i];
        *e1 = it.task_e[2 * i + 1];
    } else {
        *e0 = it.row_ptr[i];
        *e1 = it.row_ptr[i + 1];
    }
}

template <int Ls, int Ld, int UPT>
__global__ void __launch_bounds__(kBulkThreads, 1)
gather_bulk_kernel(BulkItems it, const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int64_t R,
                   uint64_t *__restrict__ out, int NS, int *err)
{
    static_assert(Ls == 1 || Ls == 2, "16-byte units hold whole values only for 1 or 2 limbs");
    constexpr int VPU = 2 / Ls;                                // values per 16-byte unit
    constexpr int NCT = kBulkConsumers * 32;                   // consumer threads
    // units per chunk and per stage: one chunk covers short rows whole, so a
    // slot is only as large as the row segment it holds
    const int64_t CHU = min((int64_t)NCT * UPT, R * Ls / 2);
    extern __shared__ __align__(128) unsigned char bulk_smem[];
    __shared__ __align__(8) uint64_t full_bar[kBulkMaxStages], empty_bar[kBulkMaxStages];
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t units = R * Ls / 2;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], kBulkConsumers);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int64_t ia, ib;
    bulk_item_range(it, &ia, &ib);
    ulonglong2 *stage = reinterpret_cast<ulonglong2 *>(bulk_smem);
    const ulonglong2 *Xv = reinterpret_cast<const ulonglong2 *>(X);
    const bool light = it.mode == 0;

    if (warp == kBulkConsumers) {
        // ---------------- producer warp: lane 0 issues, all lanes fetch ids
        int slot = 0;
        uint32_t phase = 0;
        int64_t issued = 0;
        bool ok = true;
        int64_t wbase = -64;  // window of 32 neighbour ids held one per lane
        int32_t wval = 0;
        for (int64_t ig = ia; ig < ib && ok; ig += 32) {
            const int nin = (ib - ig < 32) ? (int)(ib - ig) : 32;
            int64_t la = 0, lb = 0;
            if (lane < nin) bulk_item_load(it, ig + lane, &la, &lb);
            for (int j = 0; j < nin && ok; j++) {
                const int64_t e0 = __shfl_sync(0xffffffffu, la, j), e1 = __shfl_sync(0xffffffffu, lb, j);
                if (light && e1 - e0 > it.split) continue;
                for (int64_t cu0 = 0; cu0 < units && ok; cu0 += CHU) {
                    const uint32_t bytes = (uint32_t)(min(CHU, units - cu0) * 16);
                    for (int64_t e = e0; e < e1; e++) {
                        if (e < wbase || e >= wbase + 32) {
                            wbase = e;
                            wval = (wbase + lane < it.nnz) ? col_idx[wbase + lane] : 0;
                        }
                        const int64_t u = __shfl_sync(0xffffffffu, wval, (int)(e - wbase));
                        int good = 1;
                        if (lane == 0) {
                            good = mbar_wait(&empty_bar[slot], phase ^ 1u, err, 1) && !*((volatile int *)&abort_flag);
                            if (good) {
                                mbar_expect_tx(&full_bar[slot], bytes);
                                bulk_g2s(stage + (int64_t)slot * CHU, Xv + u * units + cu0, bytes, &full_bar[slot]);
                            }
                        }
                        if (!__shfl_sync(0xffffffffu, good, 0)) {
                            ok = false;
                            break;
                        }
                        issued++;
                        if (++slot == NS) {
                            slot = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
        }
        if (!ok && lane == 0) {
            abort_flag = 1;
            // drain: wait (bounded) for the last copy issued into each slot; slots are
            // used round-robin, so slot s received issued / NS + (s < issued % NS) copies
            for (int s = 0; s < NS; s++) {
                const int64_t cnt = issued / NS + (s < issued % NS ? 1 : 0);
                if (cnt > 0) mbar_wait(&full_bar[s], (uint32_t)((cnt - 1) & 1), err, 3);
            }
        }
    } else {
        // ---------------- consumer warps: thread t owns units t + q * NCT of a chunk
        const int t = threadIdx.x;
        int slot = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int64_t ig = ia; ig < ib && ok; ig += 32) {
            const int nin = (ib - ig < 32) ? (int)(ib - ig) : 32;
            int64_t la = 0, lb = 0;
            if (lane < nin) bulk_item_load(it, ig + lane, &la, &lb);
            for (int j = 0; j < nin && ok; j++) {
                const int64_t e0 = __shfl_sync(0xffffffffu, la, j), e1 = __shfl_sync(0xffffffffu, lb, j);
                if (light && e1 - e0 > it.split) continue;
                const int64_t orow = (ig + j) - (light ? it.v0 : it.t0);
                uint64_t *dst = out + orow * R * Ld;
                for (int64_t cu0 = 0; cu0 < units && ok; cu0 += CHU) {
                    const int64_t nun = min(CHU, units - cu0);
                    Wide<Ld> acc[UPT][VPU];
#pragma unroll
                    for (int q = 0; q < UPT; q++)
#pragma unroll
                        for (int h = 0; h < VPU; h++) wzero(acc[q][h]);
                    for (int64_t e = e0; e < e1; e++) {
                        // every lane waits on the barrier itself (acquire of the bulk-copy data)
                        const int good = mbar_wait(&full_bar[slot], phase, err, 2) && !*((volatile int *)&abort_flag);
                        if (!__all_sync(0xffffffffu, good)) {
                            ok = false;
                            break;
                        }
                        const ulonglong2 *sg = stage + (int64_t)slot * CHU;
                        ulonglong2 x[UPT];
#pragma unroll
                        for (int q = 0; q < UPT; q++) {
                            const int64_t w = t + q * NCT;
                            x[q] = (w < nun) ? sg[w] : make_ulonglong2(0, 0);
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty_bar[slot]);
#pragma unroll
                        for (int q = 0; q < UPT; q++) {
                            if constexpr (Ls == 1) {
                                Wide<Ld> a, b;
                                wzero(a);
                                wzero(b);
                                a.w[0] = x[q].x;
                                b.w[0] = x[q].y;
                                wadd(acc[q][0], a);
                                wadd(acc[q][VPU - 1], b);
                            } else {
                                Wide<Ld> a;
                                wzero(a);
                                a.w[0] = x[q].x;
                                if constexpr (Ld >= 2) a.w[1] = x[q].y;
                                wadd(acc[q][0], a);
                            }
                        }
                        if (++slot == NS) {
                            slot = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
#pragma unroll
                    for (int q = 0; q < UPT; q++) {
                        const int64_t w = t + q * NCT;
                        if (w < nun)
#pragma unroll
                            for (int h = 0; h < VPU; h++) wstore(dst + ((cu0 + w) * VPU + h) * Ld, acc[q][h]);
                    }
                }
            }
        }
        if (!ok && lane == 0) abort_flag = 1;
    }
    __syncthreads();
}

// Vectorised warp gather for rows stored with 1 or 2 limbs: the row is a run of
// 16-byte units (two 1-limb values or one 2-limb value); lane `lane` owns units
// base + lane + 32 q (q < UPT), and NB neighbours' units are loaded before any
// is added, so NB * UPT 16-byte loads per lane are in flight.
template <int Ls, int Ld, int UPT, int NB>
__device__ __forceinline__ void gather_row_vec(const int32_t *__restrict__ col_idx, int64_t e0, int64_t e1,
                                               const uint64_t *__restrict__ X, int64_t R,
                                               uint64_t *__restrict__ out_row, int lane)
{
    static_assert(Ls == 1 || Ls == 2, "16-byte units hold whole values only for 1 or 2 limbs");
    constexpr int VPU = 2 / Ls;  // values per unit
    const int64_t units = R * Ls / 2;
    const ulonglong2 *__restrict__ Xv = reinterpret_cast<const ulonglong2 *>(X);
    for (int64_t base = 0; base < units; base += 32 * UPT) {
        Wide<Ld> acc[UPT][VPU];
#pragma unroll
        for (int q = 0; q < UPT; q++)
#pragma unroll
            for (int h = 0; h < VPU; h++) wzero(acc[q][h]);
        for (int64_t e = e0; e < e1; e += 32) {
            const int cnt = (e1 - e < 32) ? (int)(e1 - e) : 32;
            const int32_t myu = lane < cnt ? col_idx[e + lane] : 0;
            for (int t = 0; t < cnt; t += NB) {
                ulonglong2 x[NB][UPT];
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    const int64_t u = __shfl_sync(0xffffffffu, myu, t + j < cnt ? t + j : t);
                    const ulonglong2 *row = Xv + u * units;
#pragma unroll
                    for (int q = 0; q < UPT; q++) {
                        const int64_t w = base + q * 32 + lane;
                        x[j][q] = (w < units && t + j < cnt) ? __ldg(row + w) : make_ulonglong2(0, 0);
                    }
                }
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    if (t + j >= cnt) break;
#pragma unroll
                    for (int q = 0; q < UPT; q++) {
                        if constexpr (Ls == 1) {
                            Wide<Ld> a, b;
                            wzero(a);
                            wzero(b);
                            a.w[0] = x[j][q].x;
                            b.w[0] = x[j][q].y;
                            wadd(acc[q][0], a);
                            wadd(acc[q][VPU - 1], b);
                        } else {
                            Wide<Ld> a;
                            wzero(a);
                            a.w[0] = x[j][q].x;
                            if constexpr (Ld >= 2) a.w[1] = x[j][q].y;
                            wadd(acc[q][0], a);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < UPT; q++) {
            const int64_t w = base + q * 32 + lane;
            if (w < units)
#pragma unroll
                for (int h = 0; h < VPU; h++) wstore(out_row + (w * VPU + h) * Ld, acc[q][h]);
        }
    }
}

template <int Ls, int Ld, int UPT, int NB>
__global__ void __launch_bounds__(kWarps * 32)
gather_light_vec_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                        const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int64_t R,
                        uint64_t *__restrict__ agg)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t v = v0 + blockIdx.x * (int64_t)kWarps + warp;
    if (v >= v1) return;
    const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
    if (e1 - e0 > split) return;  // heavy vertex: handled by tasks
    gather_row_vec<Ls, Ld, UPT, NB>(col_idx, e0, e1, X, R, agg + (v - v0) * R * Ld, lane);
}

template <int Ls, int Ld, int UPT, int NB>
__global__ void __launch_bounds__(kWarps * 32)
gather_tasks_vec_kernel(int64_t t0, int64_t t1, const int32_t *__restrict__ col_idx,
                        const int64_t *__restrict__ task_e, const uint64_t *__restrict__ X, int64_t R,
                        uint64_t *__restrict__ partial)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = t0 + blockIdx.x * (int64_t)kWarps + warp;
    if (t >= t1) return;
    gather_row_vec<Ls, Ld, UPT, NB>(col_idx, task_e[2 * t], task_e[2 * t + 1], X, R, partial + (t - t0) * R * Ld,
                                    lane);
}

// Group gather: a group of G threads (G = 32..256, a whole number of warps)
// covers a row's 16-byte units in one pass (thread gt owns units gt + G q,
// q < UPT), so even a vertex with one neighbour has its whole row in flight;
// NB neighbours are loaded before adding.  Each warp of the group fetches the
// neighbour ids itself (32 per load) and broadcasts them with shuffles.
template <int Ls, int Ld, int UPT, int NB>
__global__ void __launch_bounds__(256)
gather_group_kernel(int64_t a, int64_t b, int G, int tasks, int64_t split, const int64_t *__restrict__ row_ptr,
                    const int64_t *__restrict__ task_e, const int32_t *__restrict__ col_idx,
                    const uint64_t *__restrict__ X, int64_t R, uint64_t *__restrict__ out)
{
    static_assert(Ls == 1 || Ls == 2, "16-byte units hold whole values only for 1 or 2 limbs");
    constexpr int VPU = 2 / Ls;
    const int gpc = blockDim.x / G;
    const int grp = threadIdx.x / G, gt = threadIdx.x - grp * G, lane = threadIdx.x & 31;
    const int64_t item = a + (int64_t)blockIdx.x * gpc + grp;
    if (item >= b) return;  // whole groups (whole warps) leave together
    int64_t e0, e1;
    if (tasks) {
        e0 = task_e[2 * item];
        e1 = task_e[2 * item + 1];
    } else {
        e0 = row_ptr[item];
        e1 = row_ptr[item + 1];
        if (e1 - e0 > split) return;  // heavy vertex: handled by tasks
    }
    const int64_t units = R * Ls / 2;
    const ulonglong2 *__restrict__ Xv = reinterpret_cast<const ulonglong2 *>(X);
    uint64_t *out_row = out + (item - a) * R * Ld;
    for (int64_t base = 0; base < units; base += (int64_t)G * UPT) {
        Wide<Ld> acc[UPT][VPU];
#pragma unroll
        for (int q = 0; q < UPT; q++)
#pragma unroll
            for (int h = 0; h < VPU; h++) wzero(acc[q][h]);
        for (int64_t e = e0; e < e1; e += 32) {
            const int cnt = (e1 - e < 32) ? (int)(e1 - e) : 32;
            const int32_t myu = lane < cnt ? col_idx[e + lane] : 0;
            // one warp of the group requests the batch's rows into L2 whole
            if (base == 0 && gt < 32 && lane < cnt) prefetch_l2(Xv + (int64_t)myu * units, (uint32_t)(units * 16));
            for (int t = 0; t < cnt; t += NB) {
                ulonglong2 x[NB][UPT];
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    const int64_t u = __shfl_sync(0xffffffffu, myu, t + j < cnt ? t + j : t);
                    const ulonglong2 *row = Xv + u * units;
#pragma unroll
                    for (int q = 0; q < UPT; q++) {
                        const int64_t w = base + gt + (int64_t)q * G;
                        x[j][q] = (w < units && t + j < cnt) ? __ldg(row + w) : make_ulonglong2(0, 0);
                    }
                }
#pragma unroll
                for (int j = 0; j < NB; j++) {
#pragma unroll
                    for (int q = 0; q < UPT; q++) {
                        if constexpr (Ls == 1) {
                            Wide<Ld> lo, hi;
                            wzero(lo);
                            wzero(hi);
                            lo.w[0] = x[j][q].x;
                            hi.w[0] = x[j][q].y;
                            wadd(acc[q][0], lo);
                            wadd(acc[q][VPU - 1], hi);
                        } else {
                            Wide<Ld> v;
                            wzero(v);
                            v.w[0] = x[j][q].x;
                            if constexpr (Ld >= 2) v.w[1] = x[j][q].y;
                            wadd(acc[q][0], v);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < UPT; q++) {
            const int64_t w = base + gt + (int64_t)q * G;
            if (w < units)
#pragma unroll
                for (int h = 0; h < VPU; h++) wstore(out_row + (w * VPU + h) * Ld, acc[q][h]);
        }
    }
}

// Warp per row.  With `next` == nullptr warp w of the grid takes item w (one
// pass); otherwise the grid is persistent and each warp pulls its next item
// from the counter, so a warp that finishes a short neighbour list starts the
// next item at once instead of idling until its CTA's longest list is done.
// Persistent mode (next != nullptr): work items are (column segment, group of
// G consecutive vertices), segment-major: item i is segment i / ngroups of
// group i % ngroups.  Warps in flight then read the same segment of their
// neighbours' rows, so the segments of hub rows stay in L2 (column blocking);
// nch = G = 1 is a warp per whole row.
template <int Ls, int Ld, int VPT, bool PF = false, int NB = 2>
__global__ void __launch_bounds__(kWarps * 32)
gather_light_kernel(int64_t v0, int64_t v1, int64_t split, const int64_t *__restrict__ row_ptr,
                    const int32_t *__restrict__ col_idx, const uint64_t *__restrict__ X, int64_t R,
                    uint64_t *__restrict__ agg, unsigned long long *next, int nch, int G, AbsentSkip sk)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!next) {
        const int64_t v = v0 + blockIdx.x * (int64_t)kWarps + warp;
        if (v >= v1) return;
        const int64_t e0 = row_ptr[v], e1 = row_ptr[v + 1];
        if (e1 - e0 <= split)  // heavy vertices are summed from their tasks
            gather_row<Ls, Ld, VPT, PF, NB>(col_idx, e0, e1, X, R, agg + (v - v0) * R * Ld, lane, sk);
        return;
    }
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
            if (e1 - e0 > split) continue;
            if (nch == 1)
                gather_row<Ls, Ld, VPT, PF, NB>(col_idx, e0, e1, X, R, agg + (v - v0) * R * Ld, lane, sk);
            else
                gather_row_range<Ls, Ld, VPT, NB>(col_idx, e0, e1, X, R, seg * cw, min(R, (seg + 1) * cw),
                                                  agg + (v - v0) * R * Ld, lane, sk);
        }
    }
}

// Persistent mode (next != nullptr) runs items i in [0, nch * (t1 - t0)):
// segment i / (t1 - t0) of task t0 + i % (t1 - t0), segment-major, so the
// warps in flight read the same column segment of their neighbour rows and the
// hub rows' segments stay in L2 (column blocking).
template <int Ls, int Ld, int VPT, bool PF = false, int NB = 2>
__global__ void __launch_bounds__(kWarps * 32)
gather_tasks_kernel(int64_t t0, int64_t t1, const int32_t *__restrict__ col_idx,
                    const int64_t *__restrict__ task_e, const uint64_t *__restrict__ X, int64_t R,
                    uint64_t *__restrict__ partial, unsigned long long *next, int nch, AbsentSkip sk)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!next) {
        const int64_t t = t0 + blockIdx.x * (int64_t)kWarps + warp;
        if (t < t1)
            gather_row<Ls, Ld, VPT, PF, NB>(col_idx, task_e[2 * t], task_e[2 * t + 1], X, R,
                                            partial + (t - t0) * R * Ld, lane, sk);
        return;
    }
    const int64_t nt = t1 - t0, cw = segment_width<VPT>(R, nch);
    while (true) {
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(next, 1ull);
        const int64_t i = (int64_t)__shfl_sync(0xffffffffu, got, 0);
        if (i >= nt * nch) return;
        const int64_t seg = i / nt, t = t0 + (i - seg * nt);
        if (nch == 1)
            gather_row<Ls, Ld, VPT, PF, NB>(col_idx, task_e[2 * t], task_e[2 * t + 1], X, R,
                                            partial + (t - t0) * R * Ld, lane, sk);
        else
            gather_row_range<Ls, Ld, VPT, NB>(col_idx, task_e[2 * t], task_e[2 * t + 1], X, R, seg * cw,
                                              min(R, (seg + 1) * cw), partial + (t - t0) * R * Ld, lane, sk);
    }
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

template <int L, bool HIST>
__global__ void combine_select_kernel(int64_t total, int64_t v0, int B, int k, int64_t Ch, int64_t Chs, int64_t Cps,
                                      const uint16_t *__restrict__ rm, const uint8_t *__restrict__ col,
                                      const void *__restrict__ aggp, uint64_t *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = i / Chs, s = i - vb * Chs;
        Wide<L> x;
        wzero(x);
        if (s < Ch) {
            const int64_t lv = vb / B;
            const int b = (int)(vb - lv * B);
            const int c = col[(v0 + lv) * B + b];
            const uint32_t r = rm[s * k + c];
            if (r != 0xFFFFu) {
                if constexpr (HIST) {
                    x.w[0] = reinterpret_cast<const uint32_t *>(aggp)[vb * k + r];
                } else {
                    x = wload<L, L>(reinterpret_cast<const uint64_t *>(aggp) + (vb * Cps + r) * L);
                }
            }
        }
        wstore(out + i * L, x);
    }
}

// p = 1: out[S] = sum over c in S of act[S \ {c}] * hist[c].  The h members of S
// come from the (h, h-1) split table: entry q of S is rank(S \ {c}) | c << 16
// (the colex rank of {c} is c), laid out [q][S] so a warp reads it coalesced.
// a = 1 combine for the heavy vertices h0..h1 of the heavy list only (their
// aggregates come from the task path).
template <int L>
__global__ void select_heavy_kernel(int64_t h0, int64_t h1, int64_t v0, const int32_t *__restrict__ heavy_v, int B,
                                    int k, int64_t Ch, int64_t Chs, int64_t Cps, const uint16_t *__restrict__ rm,
                                    const uint8_t *__restrict__ col, const uint64_t *__restrict__ agg,
                                    uint64_t *__restrict__ out)
{
    const int64_t per = (int64_t)B * Chs;
    const int64_t total = (h1 - h0) * per;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hi = h0 + i / per, j = i % per;
        const int64_t v = heavy_v[hi];
        const int64_t b = j / Chs, s = j - b * Chs;
        Wide<L> x;
        wzero(x);
        if (s < Ch) {
            const uint32_t r = rm[s * k + col[v * B + b]];
            if (r != 0xFFFFu) x = wload<L, L>(agg + ((v - v0) * B * Cps + b * Cps + r) * L);
        }
        wstore(out + ((v - v0) * per + j) * L, x);
    }
}

// act rows hold La-limb values (La <= L)
template <int L, int La>
__global__ void combine_hist_kernel(int64_t rows, int k, int64_t Ch, int64_t Chs, int64_t Cas, int h,
                                    const uint32_t *__restrict__ pairs, const uint64_t *__restrict__ act,
                                    const uint32_t *__restrict__ hist, uint64_t *__restrict__ out,
                                    const uint8_t *__restrict__ cv, const uint16_t *__restrict__ rm_h,
                                    const uint16_t *__restrict__ elig, int64_t E)
{
    // zeros at the sets without the row's vertex colour and in the padding,
    // then the E outputs per row that hold it (the act rows are zero at sets
    // without it: the rooted subtree contains the vertex)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * Chs; i += stride) {
        const int64_t vb = i / Chs, s = i - vb * Chs;
        if (s >= Ch || rm_h[s * k + cv[vb]] == 0xFFFFu) {
            Wide<L> z;
            wzero(z);
            wstore(out + i * L, z);
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * E; i += stride) {
        const int64_t vb = i / E, e = i - vb * E;
        const int c = cv[vb];
        const int64_t s = elig[(int64_t)c * E + e];
        Wide<L> acc;
        wzero(acc);
        const uint64_t *ar = act + vb * Cas * La;
        const uint32_t *hr = hist + vb * k;
#pragma unroll 4
        for (int q = 0; q < h; q++) {
            const uint32_t pq = __ldg(pairs + q * Ch + s);
            const uint32_t hc = (int)(pq >> 16) == c ? 0u : hr[pq >> 16];  // S \ {col(v)} lacks col(v)
            if (hc) wmac_small(acc, wload<La, L>(ar + (pq & 0xFFFFu) * La), hc);
        }
        wstore(out + (vb * Chs + s) * L, acc);
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

// Graph batches: totals[i][b] += sum of root[v][b] over the compact vertices
// v of member graph i inside the block [v0, v1) (members hold consecutive
// compact ids, member_act[i] .. member_act[i + 1]).  One CTA per member at a
// time; CTAs stride over the members.
template <int L>
__global__ void member_reduce_kernel(int64_t v0, int64_t v1, int B, const uint64_t *__restrict__ root,
                                     const int64_t *__restrict__ member_act, int n_members,
                                     uint64_t *__restrict__ totals)
{
    for (int i = blockIdx.x; i < n_members; i += gridDim.x) {
        const int64_t a = max(v0, member_act[i]), z = min(v1, member_act[i + 1]);
        if (a >= z) continue;  // the same for every thread of the CTA
        for (int b = 0; b < B; b++) {
            Wide<L> acc;
            wzero(acc);
            for (int64_t v = a + threadIdx.x; v < z; v += blockDim.x)
                wadd(acc, wload<L, L>(root + ((v - v0) * B + b) * L));
            Wide<L> s = block_sum(acc);
            if (threadIdx.x == 0) {
                Wide<L> t;
#pragma unroll
                for (int l = 0; l < L; l++) t.w[l] = totals[((int64_t)i * B + b) * L + l];
                wadd(t, s);
                wstore(totals + ((int64_t)i * B + b) * L, t);
            }
        }
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
                                double *__restrict__ H, double *__restrict__ F)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t v = blockIdx.x * (int64_t)kWarps + warp;
    if (v >= n_act) return;
    double s = 0;
    for (int64_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) s += Hc ? Hc[col_idx[e]] : 1.0;
#pragma unroll
    for (int d = 16; d; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) {
        H[v] *= s;
        if (F) F[v] = s;
    }
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

// the colour of every list entry's neighbour in the pass's one colouring
__global__ void neighbour_colours_kernel(int64_t nnz, const int32_t *__restrict__ col_idx,
                                         const uint8_t *__restrict__ col, uint8_t *__restrict__ ncol)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        ncol[e] = col[col_idx[e]];
}

// labelled templates: rows of vertices whose label is not `want` become zero
__global__ void mask_rows_kernel(int64_t nv, int64_t row_words, const uint8_t *__restrict__ labels, int want,
                                 uint64_t *__restrict__ rows)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv * row_words;
         i += (int64_t)gridDim.x * blockDim.x)
        if (labels[i / row_words] != want) rows[i] = 0;
}

__global__ void remap_kernel(int64_t nnz, int64_t n, const int32_t *__restrict__ src,
                             const int32_t *__restrict__ new_id, int32_t *__restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nnz) {
        const int32_t u = src[i];
        dst[i] = (u >= 0 && u < n) ? new_id[u] : 0;  // ids outside [0, n) only without CC_VALIDATE
    }
}

// warp per new vertex: copies its neighbour list from the input CSR to the
// relabelled CSR, mapping every neighbour id through new_id
__global__ void permute_lists_kernel(int64_t n_act, int64_t n, const int64_t *__restrict__ orig,
                                     const int64_t *__restrict__ old_rp, const int64_t *__restrict__ new_rp,
                                     const int32_t *__restrict__ src, const int32_t *__restrict__ new_id,
                                     int32_t *__restrict__ dst)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nv = blockIdx.x * (int64_t)kWarps + warp;
    if (nv >= n_act) return;
    const int64_t ov = orig[nv];
    const int64_t a = old_rp[ov], len = old_rp[ov + 1] - a, b = new_rp[nv];
    for (int64_t i = lane; i < len; i += 32) {
        const int32_t u = src[a + i];
        dst[b + i] = (u >= 0 && u < n) ? new_id[u] : 0;  // ids outside [0, n) only without CC_VALIDATE
    }
}

template <int Ls, int Ld>
void gather_light_t(cudaStream_t st, bool pf, int nb, int64_t v0, int64_t v1, int64_t split, const int64_t *rp,
                    const int32_t *ci, const uint64_t *X, int64_t R, uint64_t *agg, unsigned long long *next, int nch,
                    int G, AbsentSkip sk)
{
    constexpr int VPT = Ld <= 2 ? 4 : 2;
    auto k = pf ? gather_light_kernel<Ls, Ld, VPT, true, 2>
                : (nb == 4 ? gather_light_kernel<Ls, Ld, VPT, false, 4> : gather_light_kernel<Ls, Ld, VPT, false, 2>);
    if (!next || pf) nch = G = 1;
    const int64_t items = (v1 - v0 + G - 1) / G * nch;
    const unsigned g = next ? std::min<unsigned>(persistent_ctas(k), grid_for(items, kWarps)) : grid_for(v1 - v0, kWarps);
    note_launch("gather_light_kernel", Ls, Ld);
    k<<<g, kWarps * 32, 0, st>>>(v0, v1, split, rp, ci, X, R, agg, next, nch, G, sk);
}

template <int Ls, int Ld>
void gather_tasks_t(cudaStream_t st, bool pf, int nb, int64_t t0, int64_t t1, const int32_t *ci, const int64_t *te,
                    const uint64_t *X, int64_t R, uint64_t *partial, unsigned long long *next, int nch,
                    AbsentSkip sk)
{
    constexpr int VPT = Ld <= 2 ? 4 : 2;
    auto k = pf ? gather_tasks_kernel<Ls, Ld, VPT, true, 2>
                : (nb == 4 ? gather_tasks_kernel<Ls, Ld, VPT, false, 4> : gather_tasks_kernel<Ls, Ld, VPT, false, 2>);
    if (!next || pf) nch = 1;
    const int64_t items = (t1 - t0) * nch;
    const unsigned g = next ? std::min<unsigned>(persistent_ctas(k), grid_for(items, kWarps)) : grid_for(t1 - t0, kWarps);
    note_launch("gather_tasks_kernel", Ls, Ld);
    k<<<g, kWarps * 32, 0, st>>>(t0, t1, ci, te, X, R, partial, next, nch, sk);
}

}  // namespace

namespace {
thread_local std::vector<std::string> t_launch_names;
}

void note_launch(const char *kernel, int a, int b, int c)
{
    std::string s(kernel);
    if (a >= 0) {
        s += "<" + std::to_string(a);
        if (b >= 0) s += "," + std::to_string(b);
        if (c >= 0) s += "," + std::to_string(c);
        s += ">";
    }
    t_launch_names.push_back(std::move(s));
}

std::vector<std::string> take_launch_names()
{
    std::vector<std::string> r;
    r.swap(t_launch_names);
    return r;
}

void launch_colour(cudaStream_t st, int64_t n_act, int B, int k, const int64_t *orig_id,
                   const ColourParams *prm, uint8_t *col)
{
    if (n_act == 0) return;
    colour_kernel<<<grid_for(n_act * B, 256), 256, 0, st>>>(n_act, B, k, orig_id, prm, col);
}

void launch_hist(cudaStream_t st, int64_t v0, int64_t v1, int B, int k, const int64_t *row_ptr,
                 const int32_t *col_idx, const uint8_t *col, uint32_t *hist, const uint8_t *labels, int want)
{
    if (v1 <= v0) return;
    size_t sh = (size_t)kWarps * B * k * sizeof(uint32_t);
    hist_kernel<<<grid_for(v1 - v0, kWarps), kWarps * 32, sh, st>>>(v0, v1, B, k, row_ptr, col_idx, col, labels, want,
                                                                  hist);
}

void launch_neighbour_colours(cudaStream_t st, int64_t nnz, const int32_t *col_idx, const uint8_t *col,
                              uint8_t *ncol)
{
    if (nnz <= 0) return;
    note_launch("neighbour_colours_kernel");
    neighbour_colours_kernel<<<grid_stride_ctas(nnz, 256), 256, 0, st>>>(nnz, col_idx, col, ncol);
}

void launch_mask_rows(cudaStream_t st, int64_t nv, int64_t row_words, const uint8_t *labels, int want, uint64_t *rows)
{
    if (nv <= 0 || row_words <= 0) return;
    mask_rows_kernel<<<grid_stride_ctas(nv * row_words, 256), 256, 0, st>>>(nv, row_words, labels, want, rows);
}

void launch_gather_light(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                         const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int64_t R,
                         uint64_t *agg, bool prefetch, unsigned long long *next, int nb, int nch, int G,
                         AbsentSkip sk)
{
    if (v1 <= v0) return;
    nch = std::max(1, std::min(nch, 64));
    G = std::max(1, G);
#define CC_GL(a, b) if (Ls == a && Ld == b) return gather_light_t<a, b>(st, prefetch, nb, v0, v1, split, row_ptr, col_idx, X, R, agg, next, nch, G, sk)
    CC_GL(1, 1); CC_GL(1, 2); CC_GL(1, 3); CC_GL(1, 4);
    CC_GL(2, 1); CC_GL(2, 2); CC_GL(2, 3); CC_GL(2, 4);
    CC_GL(3, 1); CC_GL(3, 2); CC_GL(3, 3); CC_GL(3, 4);
    CC_GL(4, 1); CC_GL(4, 2); CC_GL(4, 3); CC_GL(4, 4);
#undef CC_GL
}

namespace {

template <int Ls, int Ld>
void gather_bulk_t(cudaStream_t st, const BulkItems &it, const int32_t *ci, const uint64_t *X, int64_t R,
                   uint64_t *out, int *err)
{
    constexpr int UPT = 2;
    const int64_t stage_bytes = std::min<int64_t>((int64_t)kBulkConsumers * 32 * UPT, R * Ls / 2) * 16;
    const int NS = (int)std::max<int64_t>(2, std::min<int64_t>(kBulkMaxStages, kBulkSmemBytes / stage_bytes));
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    gather_bulk_kernel<Ls, Ld, UPT><<<sms, kBulkThreads, (size_t)NS * stage_bytes, st>>>(it, ci, X, R, out, NS, err);
}

void gather_bulk_dispatch(cudaStream_t st, int Ls, int Ld, const BulkItems &it, const int32_t *ci,
                          const uint64_t *X, int64_t R, uint64_t *out, int *err)
{
#define CC_GB(a, b) if (Ls == a && Ld == b) return gather_bulk_t<a, b>(st, it, ci, X, R, out, err)
    CC_GB(1, 1); CC_GB(1, 2); CC_GB(1, 3); CC_GB(1, 4);
    CC_GB(2, 1); CC_GB(2, 2); CC_GB(2, 3); CC_GB(2, 4);
#undef CC_GB
}

template <int Ls, int Ld>
void gather_vec_t(cudaStream_t st, bool tasks, int64_t a, int64_t b, int64_t split, const int64_t *rp,
                  const int32_t *ci, const int64_t *te, const uint64_t *X, int64_t R, uint64_t *out)
{
    constexpr int UPT = 4, NB = 4;
    if (tasks)
        gather_tasks_vec_kernel<Ls, Ld, UPT, NB><<<grid_for(b - a, kWarps), kWarps * 32, 0, st>>>(a, b, ci, te, X, R,
                                                                                                  out);
    else
        gather_light_vec_kernel<Ls, Ld, UPT, NB><<<grid_for(b - a, kWarps), kWarps * 32, 0, st>>>(a, b, split, rp, ci,
                                                                                                  X, R, out);
}

void gather_vec_dispatch(cudaStream_t st, bool tasks, int Ls, int Ld, int64_t a, int64_t b, int64_t split,
                         const int64_t *rp, const int32_t *ci, const int64_t *te, const uint64_t *X, int64_t R,
                         uint64_t *out)
{
#define CC_GV(x, y) if (Ls == x && Ld == y) return gather_vec_t<x, y>(st, tasks, a, b, split, rp, ci, te, X, R, out)
    CC_GV(1, 1); CC_GV(1, 2); CC_GV(1, 3); CC_GV(1, 4);
    CC_GV(2, 1); CC_GV(2, 2); CC_GV(2, 3); CC_GV(2, 4);
#undef CC_GV
}

}  // namespace

namespace {

template <int Ls, int Ld>
void gather_group_t(cudaStream_t st, bool tasks, int64_t a, int64_t b, int64_t split, const int64_t *rp,
                    const int64_t *te, const int32_t *ci, const uint64_t *X, int64_t R, uint64_t *out)
{
    constexpr int UPT = 4, NB = 2;
    const int64_t units = R * Ls / 2;
    int G = 32;
    while (G < 256 && (int64_t)G * UPT < units) G <<= 1;
    const int gpc = 256 / G;
    gather_group_kernel<Ls, Ld, UPT, NB><<<grid_for(b - a, gpc), 256, 0, st>>>(a, b, G, tasks ? 1 : 0, split, rp, te,
                                                                              ci, X, R, out);
}

void gather_group_dispatch(cudaStream_t st, bool tasks, int Ls, int Ld, int64_t a, int64_t b, int64_t split,
                           const int64_t *rp, const int64_t *te, const int32_t *ci, const uint64_t *X, int64_t R,
                           uint64_t *out)
{
#define CC_GG(x, y) if (Ls == x && Ld == y) return gather_group_t<x, y>(st, tasks, a, b, split, rp, te, ci, X, R, out)
    CC_GG(1, 1); CC_GG(1, 2); CC_GG(1, 3); CC_GG(1, 4);
    CC_GG(2, 1); CC_GG(2, 2); CC_GG(2, 3); CC_GG(2, 4);
#undef CC_GG
}

}  // namespace

void launch_gather_light_group(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                               const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int64_t R,
                               uint64_t *agg)
{
    if (v1 <= v0) return;
    gather_group_dispatch(st, false, Ls, Ld, v0, v1, split, row_ptr, nullptr, col_idx, X, R, agg);
}

void launch_gather_tasks_group(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                               const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial)
{
    if (t1 <= t0) return;
    gather_group_dispatch(st, true, Ls, Ld, t0, t1, 0, nullptr, task_e, col_idx, X, R, partial);
}

bool vec_gather_ok(int Ls, int64_t R) { return (Ls == 1 || Ls == 2) && (R * Ls) % 2 == 0; }

void launch_gather_light_vec(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                             const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *X, int64_t R,
                             uint64_t *agg)
{
    if (v1 <= v0) return;
    gather_vec_dispatch(st, false, Ls, Ld, v0, v1, split, row_ptr, col_idx, nullptr, X, R, agg);
}

void launch_gather_tasks_vec(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                             const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial)
{
    if (t1 <= t0) return;
    gather_vec_dispatch(st, true, Ls, Ld, t0, t1, 0, nullptr, col_idx, task_e, X, R, partial);
}

bool bulk_gather_ok(int Ls, int64_t R)
{
    // whole values per 16-byte unit, whole units per row, rows big enough to amortise a copy
    return (Ls == 1 || Ls == 2) && (R * Ls) % 2 == 0 && R * Ls * 8 >= 1024;
}

void init_kernel_attributes()
{
#define CC_ATTR(a, b)                                                                                       \
    cudaFuncSetAttribute(gather_bulk_kernel<a, b, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                         (int)kBulkSmemBytes)
    CC_ATTR(1, 1); CC_ATTR(1, 2); CC_ATTR(1, 3); CC_ATTR(1, 4);
    CC_ATTR(2, 1); CC_ATTR(2, 2); CC_ATTR(2, 3); CC_ATTR(2, 4);
#undef CC_ATTR
}

void launch_gather_light_bulk(cudaStream_t st, int Ls, int Ld, int64_t v0, int64_t v1, int64_t split,
                              const int64_t *row_ptr, const int32_t *col_idx, int64_t nnz, const uint64_t *X,
                              int64_t R, uint64_t *agg, int *err)
{
    if (v1 <= v0) return;
    BulkItems it{};
    it.mode = 0;
    it.nnz = nnz;
    it.v0 = v0;
    it.v1 = v1;
    it.split = split;
    it.row_ptr = row_ptr;
    gather_bulk_dispatch(st, Ls, Ld, it, col_idx, X, R, agg, err);
}

void launch_gather_tasks_bulk(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                              int64_t nnz, const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial,
                              int *err)
{
    if (t1 <= t0) return;
    BulkItems it{};
    it.mode = 1;
    it.nnz = nnz;
    it.t0 = t0;
    it.t1 = t1;
    it.task_e = task_e;
    gather_bulk_dispatch(st, Ls, Ld, it, col_idx, X, R, partial, err);
}

void launch_gather_tasks(cudaStream_t st, int Ls, int Ld, int64_t t0, int64_t t1, const int32_t *col_idx,
                         const int64_t *task_e, const uint64_t *X, int64_t R, uint64_t *partial, bool prefetch,
                         unsigned long long *next, int nb, int nch, AbsentSkip sk)
{
    if (t1 <= t0) return;
    nch = std::max(1, std::min(nch, 64));
#define CC_GT(a, b) if (Ls == a && Ld == b) return gather_tasks_t<a, b>(st, prefetch, nb, t0, t1, col_idx, task_e, X, R, partial, next, nch, sk)
    CC_GT(1, 1); CC_GT(1, 2); CC_GT(1, 3); CC_GT(1, 4);
    CC_GT(2, 1); CC_GT(2, 2); CC_GT(2, 3); CC_GT(2, 4);
    CC_GT(3, 1); CC_GT(3, 2); CC_GT(3, 3); CC_GT(3, 4);
    CC_GT(4, 1); CC_GT(4, 2); CC_GT(4, 3); CC_GT(4, 4);
#undef CC_GT
}

int column_segments(int64_t R, int Ls, int requested)
{
    (void)Ls;
    if (requested > 0) return std::min(requested, 64);
    // one warp sweep (32 lanes x 4 values) per segment, at most 16 segments
    return (int)std::max<int64_t>(1, std::min<int64_t>(16, (R + 127) / 128));
}

void launch_gather_reduce(cudaStream_t st, int Ld, int64_t h0, int64_t h1, int64_t v0, int64_t t0,
                          const int32_t *heavy_v, const int64_t *heavy_tptr, const uint64_t *partial, int64_t R,
                          uint64_t *agg)
{
    if (h1 <= h0) return;
    note_launch("gather_reduce_kernel", Ld);
    CC_DISPATCH_L(Ld, gather_reduce_kernel<LL><<<grid_for(h1 - h0, kWarps), kWarps * 32, 0, st>>>(
                          h0, h1, v0, t0, heavy_v, heavy_tptr, partial, R, agg));
}

void launch_combine_select(cudaStream_t st, int L, bool agg_is_hist, int64_t v0, int64_t nv, int B, int k,
                           int64_t Ch, int64_t Chs, int64_t Cps, const uint16_t *rm, const uint8_t *col,
                           const void *agg, uint64_t *out)
{
    const int64_t total = nv * B * Chs;
    if (total == 0) return;
    note_launch(agg_is_hist ? "combine_select_kernel<hist>" : "combine_select_kernel", L);
    if (agg_is_hist) {
        CC_DISPATCH_L(L, combine_select_kernel<LL, true><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                             total, v0, B, k, Ch, Chs, Cps, rm, col, agg, out));
    } else {
        CC_DISPATCH_L(L, combine_select_kernel<LL, false><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                             total, v0, B, k, Ch, Chs, Cps, rm, col, agg, out));
    }
}

void launch_combine_hist(cudaStream_t st, int L, int La, int64_t nv, int B, int k, int64_t Ch, int64_t Chs,
                         int64_t Cas, int h, const uint32_t *pairs, const uint64_t *act, const uint32_t *hist,
                         uint64_t *out, const uint8_t *cv, const uint16_t *rm_h, const uint16_t *elig, int64_t E)
{
    const int64_t total = nv * B * Chs;
    if (total == 0) return;
    L = std::max(1, std::min(L, 4));
    La = std::max(1, std::min(La, L));
    const unsigned g = grid_stride_ctas(total, 256);
    note_launch("combine_hist_kernel", L, La);
#define CC_CH(l, a)                                                                                        \
    case ((l - 1) * 4 + (a - 1)):                                                                          \
        combine_hist_kernel<l, a><<<g, 256, 0, st>>>(nv * B, k, Ch, Chs, Cas, h, pairs, act, hist, out, cv, rm_h, \
                                                     elig, E);                                                       \
        break;
    switch ((L - 1) * 4 + (La - 1)) {
        CC_CH(1, 1) CC_CH(2, 1) CC_CH(2, 2) CC_CH(3, 1) CC_CH(3, 2) CC_CH(3, 3)
        CC_CH(4, 1) CC_CH(4, 2) CC_CH(4, 3) CC_CH(4, 4)
    default: break;
    }
#undef CC_CH
}

void launch_select_heavy(cudaStream_t st, int L, int64_t h0, int64_t h1, int64_t v0, const int32_t *heavy_v, int B,
                         int k, int64_t Ch, int64_t Chs, int64_t Cps, const uint16_t *rm, const uint8_t *col,
                         const uint64_t *agg, uint64_t *out)
{
    const int64_t total = (h1 - h0) * B * Chs;
    if (total <= 0) return;
    note_launch("select_heavy_kernel", L);
    CC_DISPATCH_L(L, select_heavy_kernel<LL><<<grid_stride_ctas(total, 256), 256, 0, st>>>(
                         h0, h1, v0, heavy_v, B, k, Ch, Chs, Cps, rm, col, agg, out));
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

void launch_member_reduce(cudaStream_t st, int L, int64_t v0, int64_t v1, int B, const uint64_t *root,
                          const int64_t *member_act, int n_members, uint64_t *totals)
{
    if (v1 <= v0 || n_members <= 0) return;
    const unsigned g = (unsigned)std::min(n_members, 152 * 8);
    CC_DISPATCH_L(L, member_reduce_kernel<LL><<<g, 256, 0, st>>>(v0, v1, B, root, member_act, n_members, totals));
}

void launch_sample_extract(cudaStream_t st, int L, int64_t n_s, const int64_t *sample_v, int64_t v0, int64_t v1,
                           int B, const uint64_t *root, uint64_t *out)
{
    if (n_s == 0) return;
    CC_DISPATCH_L(L, sample_kernel<LL><<<grid_for(n_s * B, 256), 256, 0, st>>>(n_s, sample_v, v0, v1, B, root,
                                                                                out));
}

void launch_hom_step(cudaStream_t st, int64_t n_act, const int64_t *row_ptr, const int32_t *col_idx,
                     const double *Hc, double *H, double *F)
{
    if (n_act == 0) return;
    hom_step_kernel<<<grid_for(n_act, kWarps), kWarps * 32, 0, st>>>(n_act, row_ptr, col_idx, Hc, H, F);
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

void launch_permute_lists(cudaStream_t st, int64_t n_act, int64_t n, const int64_t *orig, const int64_t *old_rp,
                          const int64_t *new_rp, const int32_t *src, const int32_t *new_id, int32_t *dst)
{
    if (n_act == 0) return;
    permute_lists_kernel<<<grid_for(n_act, kWarps), kWarps * 32, 0, st>>>(n_act, n, orig, old_rp, new_rp, src,
                                                                           new_id, dst);
}

void launch_remap(cudaStream_t st, int64_t nnz, int64_t n, const int32_t *src, const int32_t *new_id, int32_t *dst)
{
    if (nnz == 0) return;
    remap_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, n, src, new_id, dst);
}

}  // namespace cc
