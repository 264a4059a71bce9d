// noalloc.cu -- the table gather for callers that cannot allocate device memory.
//
// cc_table_gather takes its task list and the tasks' partial rows from the
// context's arena, and the arena itself is a device allocation.  Some callers
// cannot make one: a host framework that owns every byte of device memory
// through its own pool and forbids side allocations, a latency-bound loop in
// which cudaMalloc/cudaFree (which may synchronise the device) are not
// acceptable, or a process handed a fixed memory budget with nothing spare.
// cc_table_gather_noalloc serves them: it runs the same three kernels (light
// rows, split-list tasks, task reduce) but keeps the task list and the partial
// rows in one file-scope device array of fixed size, so it calls no cudaMalloc,
// no cudaFree and no allocating library routine.
//
// The array costs every GPU that loads this library kNoAllocScratchBytes of
// device memory until the process exits.  All calls share it, so two calls
// whose kernels overlap on the GPU (different streams, or different host
// threads on the same device) race on it; serialise them.
#include <mutex>
#include <string>

#include "../../include/cc.h"
#include "kernels.cuh"

namespace cc {

cc_status fail(cc_status s, const std::string &msg);

namespace {

constexpr uint64_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB
constexpr int kMaxDevices = 64;
constexpr int kBuildThreads = 1024;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct Header {
    long long tasks;     // T
    long long heavy;     // H
    long long overflow;  // 1 if the lists did not fit
    long long bad_rows;  // 1 if some row_ptr[v + 1] < row_ptr[v]
};

struct Layout {
    uint64_t off_tasks, off_heavy_v, off_tptr, off_partial;
    long long max_tasks, max_heavy;
};

inline uint64_t al256(uint64_t x) { return (x + 255) / 256 * 256; }

// Space for T tasks needs 16 B (neighbour range) + one partial row each; every
// heavy vertex owns at least two tasks, so H <= T bounds the vertex lists.
bool layout_for(uint64_t row_bytes, Layout *L)
{
    const uint64_t fixed = 256 + 4 * 256 + 8;  // header, alignment slack, tptr sentinel
    if (row_bytes == 0 || fixed >= kNoAllocScratchBytes) return false;
    const uint64_t per_task = 16 + 4 + 8 + row_bytes;
    long long T = (long long)((kNoAllocScratchBytes - fixed) / per_task);
    if (T < 1) return false;
    L->max_tasks = T;
    L->max_heavy = T;
    L->off_tasks = 256;
    L->off_heavy_v = al256(L->off_tasks + 16ull * T);
    L->off_tptr = al256(L->off_heavy_v + 4ull * T);
    L->off_partial = al256(L->off_tptr + 8ull * (T + 1));
    return L->off_partial + row_bytes * (uint64_t)T <= kNoAllocScratchBytes;
}

// Exclusive scan of one value per thread over the CTA; returns the CTA total.
__device__ long long cta_exclusive_scan(long long x, long long *excl)
{
    __shared__ long long warp_tot[kBuildThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < kBuildThreads / 32 ? warp_tot[lane] : 0;
        long long wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < kBuildThreads / 32) warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    *excl = warp_tot[warp] + inc - x;
    long long total = 0;
    if (threadIdx.x == kBuildThreads - 1) total = *excl + x;
    __shared__ long long tot;
    if (threadIdx.x == kBuildThreads - 1) tot = total;
    __syncthreads();
    total = tot;
    __syncthreads();
    return total;
}

// One CTA: the split-list task list (Algorithm 4) for every vertex with more
// than `split` neighbours, written into the static scratch.  Each thread takes
// kPerThread consecutive vertices per round; a CTA-wide scan of the per-thread
// task and vertex counts gives every heavy vertex its slots.
constexpr int kPerThread = 8;

__global__ void __launch_bounds__(kBuildThreads)
noalloc_tasks_kernel(long long n, const int64_t *__restrict__ row_ptr, long long split, unsigned char *scratch,
                     Layout L)
{
    Header *hdr = reinterpret_cast<Header *>(scratch);
    int64_t *tasks = reinterpret_cast<int64_t *>(scratch + L.off_tasks);
    int32_t *heavy_v = reinterpret_cast<int32_t *>(scratch + L.off_heavy_v);
    int64_t *tptr = reinterpret_cast<int64_t *>(scratch + L.off_tptr);
    long long T = 0, H = 0;
    int overflow = 0, bad = 0;
    for (long long base = 0; base < n; base += (long long)kBuildThreads * kPerThread) {
        const long long v0 = base + (long long)threadIdx.x * kPerThread;
        long long my_t = 0, my_h = 0;
        for (int i = 0; i < kPerThread; i++) {
            const long long v = v0 + i;
            if (v >= n) break;
            const long long d = row_ptr[v + 1] - row_ptr[v];
            bad |= d < 0;
            if (d > split) {
                my_t += (d + split - 1) / split;
                my_h += 1;
            }
        }
        long long tpos, hpos;
        const long long tsum = cta_exclusive_scan(my_t, &tpos);
        const long long hsum = cta_exclusive_scan(my_h, &hpos);
        long long t_at = T + tpos, h_at = H + hpos;
        for (int i = 0; i < kPerThread && my_h > 0; i++) {
            const long long v = v0 + i;
            if (v >= n) break;
            const long long e0 = row_ptr[v], e1 = row_ptr[v + 1];
            if (e1 - e0 <= split) continue;
            const long long nt = (e1 - e0 + split - 1) / split;
            if (t_at + nt <= L.max_tasks && h_at < L.max_heavy) {
                heavy_v[h_at] = (int32_t)v;
                tptr[h_at] = t_at;
                for (long long q = 0; q < nt; q++) {
                    const long long a = e0 + q * split;
                    tasks[2 * (t_at + q)] = a;
                    tasks[2 * (t_at + q) + 1] = a + split < e1 ? a + split : e1;
                }
            } else {
                overflow = 1;
            }
            t_at += nt;
            h_at += 1;
        }
        T += tsum;
        H += hsum;
        overflow = __syncthreads_or(overflow);
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        const bool fits = !overflow && T <= L.max_tasks && H <= L.max_heavy;
        if (fits) tptr[H] = T;
        hdr->tasks = T;
        hdr->heavy = H;
        hdr->overflow = fits ? 0 : 1;
        hdr->bad_rows = bad ? 1 : 0;
    }
}

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once.
cc_status scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(CC_ERR_INVALID_ARG, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(CC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return CC_OK;
}

}  // namespace

}  // namespace cc

extern "C" cc_status cc_table_gather_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                                             const uint64_t *X, uint64_t *agg, int64_t values, int32_t limbs,
                                             int32_t split_threshold, void *stream)
{
    using namespace cc;
    if (n < 0 || n >= (int64_t(1) << 31) || values < 1 || limbs < 1 || limbs > 4 || split_threshold < 0)
        return fail(CC_ERR_INVALID_ARG, "bad n, values, limbs or split_threshold");
    if (n == 0) return CC_OK;
    if (!row_ptr || !col_idx || !X || !agg) return fail(CC_ERR_INVALID_ARG, "NULL device pointer");
    const uint64_t row_bytes = (uint64_t)values * (uint64_t)limbs * 8;
    Layout L;
    if (!layout_for(row_bytes, &L))
        return fail(CC_ERR_CAPACITY, "a row of " + std::to_string(row_bytes) + " bytes does not fit the " +
                                         std::to_string(kNoAllocScratchBytes >> 20) + " MiB static scratch");
    unsigned char *scratch = nullptr;
    cc_status rc = scratch_address(&scratch);
    if (rc != CC_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long s = split_threshold > 0 ? split_threshold : 1024;
    // every field of the header and every task/partial read later is written by this call
    noalloc_tasks_kernel<<<1, kBuildThreads, 0, st>>>(n, row_ptr, s, scratch, L);
    cudaError_t e = cudaGetLastError();
    Header hdr{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hdr, scratch, sizeof hdr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, std::string("task list: ") + cudaGetErrorString(e));
    if (hdr.bad_rows) return fail(CC_ERR_INVALID_ARG, "row_ptr decreases");
    if (hdr.overflow)
        return fail(CC_ERR_CAPACITY, "split lists need " + std::to_string(hdr.tasks) + " tasks of " +
                                         std::to_string(row_bytes) + " bytes; the static scratch holds " +
                                         std::to_string(L.max_tasks) + " (raise split_threshold)");
    launch_gather_light(st, limbs, limbs, 0, n, s, row_ptr, col_idx, X, values, agg);
    if (hdr.tasks > 0) {
        const int64_t *tasks = reinterpret_cast<const int64_t *>(scratch + L.off_tasks);
        const int32_t *heavy_v = reinterpret_cast<const int32_t *>(scratch + L.off_heavy_v);
        const int64_t *tptr = reinterpret_cast<const int64_t *>(scratch + L.off_tptr);
        uint64_t *partial = reinterpret_cast<uint64_t *>(scratch + L.off_partial);
        launch_gather_tasks(st, limbs, limbs, 0, hdr.tasks, col_idx, tasks, X, values, partial);
        launch_gather_reduce(st, limbs, 0, hdr.heavy, 0, 0, heavy_v, tptr, partial, values, agg);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(CC_ERR_CUDA, std::string("table gather: ") + cudaGetErrorString(e));
    return CC_OK;
}
