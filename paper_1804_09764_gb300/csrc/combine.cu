// combine.cu -- Eq. 1's general combine (arXiv 1804.09764, Section 2.1):
//   out[v][S] = sum over S_a u S_p = S (disjoint, |S_a| = a, |S_p| = p) of
//               act[v][S_a] * agg[v][S_p]
// for steps with a >= 2 and p >= 2, on unsigned integers modulo 2^(64 L), each
// operand read at the width its own bound needs.  (The a = 1 and p = 1 forms
// are in kernels.cu.)
#include "kernels.cuh"
#include "wideint.cuh"

#include <algorithm>

namespace cc {

namespace {

inline unsigned grid_stride_ctas(int64_t items, int threads)
{
    int64_t g = (items + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

// Every row of a chain at vertex v is zero at the colour sets without v's own
// colour col(v): the rooted subtree contains v.  So out[v][S] is zero unless
// col(v) is in S, and the combines compute only the E = C(k-1, h-1) outputs S
// that hold col(v) -- elig[c * E + e], e < E, lists the ranks of the h-sets
// holding colour c in increasing order -- and write zeros at the others
// (rm_h[S * k + c] == 0xFFFF: c not in S) and in the padding columns.  cv[vb]
// is col(v) for row vb (vertex-major, colouring-minor, like the rows).

// The sum over the npairs splits of output column s of one row, read from the
// row's act values ar (La limbs) and aggregate pr (Lb limbs), in groups of G:
// split entries, then both operands, then the multiply-adds.
template <int L, int La, int Lb, int G, typename Act, typename Agg>
__device__ __forceinline__ Wide<L> split_sum(int64_t s, int64_t Ch, int64_t npairs, const uint32_t *__restrict__ pairs,
                                             Act ar, Agg pr)
{
    Wide<L> acc;
    wzero(acc);
    const uint32_t *ps = pairs + s;
    int64_t q0 = 0;
    for (; q0 + G <= npairs; q0 += G) {
        uint32_t pq[G];
#pragma unroll
        for (int j = 0; j < G; j++) pq[j] = __ldg(ps + (q0 + j) * Ch);
#pragma unroll
        for (int j = 0; j < G; j++) {
            Wide<La> x;
            Wide<Lb> y;
#pragma unroll
            for (int l = 0; l < La; l++) x.w[l] = ar[(pq[j] & 0xFFFFu) * La + l];
#pragma unroll
            for (int l = 0; l < Lb; l++) y.w[l] = pr[(pq[j] >> 16) * Lb + l];
            wmac_mixed<L, La, Lb>(acc, x, y);
        }
    }
    for (int64_t q = q0; q < npairs; q++) {
        const uint32_t pq = __ldg(ps + q * Ch);
        Wide<La> x;
        Wide<Lb> y;
#pragma unroll
        for (int l = 0; l < La; l++) x.w[l] = ar[(pq & 0xFFFFu) * La + l];
#pragma unroll
        for (int l = 0; l < Lb; l++) y.w[l] = pr[(pq >> 16) * Lb + l];
        wmac_mixed<L, La, Lb>(acc, x, y);
    }
    return acc;
}

// Rows carry Cs >= C columns (C rounded up to even so a row is a whole number of
// 16-byte units); columns C..Cs-1 are written as zero.  act rows hold La-limb
// values, agg rows Lb-limb values, out rows L-limb values (La, Lb <= L): each
// operand is read at the width its bound needs and the product is formed only
// from the limb products below limb L.  One thread per output: first the zeros
// of every row, then the E outputs per row that hold col(v).
template <int L, int La, int Lb>
__global__ void combine_generic_kernel(int64_t rows, int64_t Ch, int64_t Chs, int64_t Cas, int64_t Cps,
                                       int64_t npairs, const uint32_t *__restrict__ pairs,
                                       const uint64_t *__restrict__ act, const uint64_t *__restrict__ agg,
                                       uint64_t *__restrict__ out, int k, const uint8_t *__restrict__ cv,
                                       const uint16_t *__restrict__ rm_h, const uint16_t *__restrict__ elig,
                                       int64_t E)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * Chs; i += stride) {
        const int64_t vb = i / Chs, s = i - vb * Chs;
        if (s >= Ch || rm_h[s * k + cv[vb]] == 0xFFFFu) {
            Wide<L> z;
            wzero(z);
            wstore(out + i * L, z);
        }
    }
    constexpr int G = L <= 1 ? 4 : 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * E; i += stride) {
        const int64_t vb = i / E, e = i - vb * E;
        const int64_t s = elig[(int64_t)cv[vb] * E + e];
        const Wide<L> acc = split_sum<L, La, Lb, G>(s, Ch, npairs, pairs, act + vb * Cas * La, agg + vb * Cps * Lb);
        wstore(out + (vb * Chs + s) * L, acc);
    }
}

// The same combine with one CTA per (vertex, colouring) row at a time: the
// row's act values (Cas x La words) and aggregate (Cps x Lb words) are staged
// in shared memory, then its threads compute the row's outputs from there.
// Used for large rows, whose random act reads would otherwise miss L1
// (several rows of ~100 KB per SM).
template <int L, int La, int Lb>
__global__ void __launch_bounds__(512)
combine_generic_smem_kernel(int64_t rows, int64_t Ch, int64_t Chs, int64_t Cas, int64_t Cps, int64_t npairs,
                            const uint32_t *__restrict__ pairs, const uint64_t *__restrict__ act,
                            const uint64_t *__restrict__ agg, uint64_t *__restrict__ out, int k,
                            const uint8_t *__restrict__ cv, const uint16_t *__restrict__ rm_h,
                            const uint16_t *__restrict__ elig, int64_t E)
{
    extern __shared__ uint64_t sm[];
    uint64_t *sa = sm, *sp = sm + Cas * La;
    for (int64_t vb = blockIdx.x; vb < rows; vb += gridDim.x) {
        __syncthreads();
        const uint64_t *ar = act + vb * Cas * La;
        const uint64_t *pr = agg + vb * Cps * Lb;
        for (int64_t i = threadIdx.x; i < Cas * La; i += blockDim.x) sa[i] = __ldg(ar + i);
        for (int64_t i = threadIdx.x; i < Cps * Lb; i += blockDim.x) sp[i] = __ldg(pr + i);
        const int c = cv[vb];
        for (int64_t s = threadIdx.x; s < Chs; s += blockDim.x)
            if (s >= Ch || rm_h[s * k + c] == 0xFFFFu) {
                Wide<L> z;
                wzero(z);
                wstore(out + (vb * Chs + s) * L, z);
            }
        __syncthreads();
        // split entries G at a time (all G global loads in flight before the
        // shared-memory operand reads and multiply-adds that need them)
        constexpr int G = L <= 2 ? 8 : 4;
        for (int64_t e = threadIdx.x; e < E; e += blockDim.x) {
            const int64_t s = elig[(int64_t)c * E + e];
            const Wide<L> acc = split_sum<L, La, Lb, G>(s, Ch, npairs, pairs, (const uint64_t *)sa,
                                                        (const uint64_t *)sp);
            wstore(out + (vb * Chs + s) * L, acc);
        }
    }
}

// Register-resident 64-bit multiply-adds as in the combines: 8 independent
// 128-bit accumulators per thread, each step one 64 x 64 -> 128-bit product
// (two limb products: low and high halves) and its carry-propagating add.
__global__ void limb_product_rate_kernel(int64_t iters, uint64_t seed, uint64_t *out)
{
    Wide<2> acc[8];
    Wide<1> x[8], y[8];
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        wzero(acc[j]);
        x[j].w[0] = seed ^ (t * 0x9E3779B97F4A7C15ull + j);
        y[j].w[0] = (seed + j) * 0xBF58476D1CE4E5B9ull | 1;
    }
    for (int64_t i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) {
            wmac_mixed<2, 1, 1>(acc[j], x[j], y[j]);
            x[j].w[0] += acc[j].w[1];  // keeps every step dependent on the last
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) r ^= acc[j].w[0] ^ acc[j].w[1];
    if (r == seed) out[0] = r;  // practically never; keeps the loop alive
}

}  // namespace

double limb_product_rate(cudaStream_t st, uint64_t *scratch)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = sms * 8;
    const int64_t iters = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    limb_product_rate_kernel<<<blocks, threads, 0, st>>>(iters / 8, 1, scratch);  // warm-up
    cudaEventRecord(a, st);
    limb_product_rate_kernel<<<blocks, threads, 0, st>>>(iters, 2, scratch);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess || ms <= 0) return 0;
    return (double)blocks * threads * iters * 8 * 2 / (ms * 1e-3);
}

void launch_combine_generic(cudaStream_t st, int L, int La, int Lb, int64_t nv, int B, int64_t Ch, int64_t Chs,
                            int64_t Cas, int64_t Cps, int64_t npairs, const uint32_t *pairs, const uint64_t *act,
                            const uint64_t *agg, uint64_t *out, int k, const uint8_t *cv, const uint16_t *rm_h,
                            const uint16_t *elig, int64_t E)
{
    const int64_t total = nv * B * Chs;
    if (total == 0) return;
    L = std::max(1, std::min(L, 4));
    La = std::max(1, std::min(La, L));
    Lb = std::max(1, std::min(Lb, L));
    const unsigned g = grid_stride_ctas(total, 256);
    // rows whose operands take at least 16 KiB are staged in shared memory
    const size_t smem = (size_t)(Cas * La + Cps * Lb) * 8;
    const bool staged = smem >= (16u << 10) && smem <= (200u << 10);
    const int64_t rows = nv * B;
    note_launch(staged ? "combine_generic_smem_kernel" : "combine_generic_kernel", L, La, Lb);
#define CC_CG(l, a, b)                                                                              \
    case ((l - 1) * 16 + (a - 1) * 4 + (b - 1)):                                                    \
        if (staged) {                                                                               \
            auto kfn = combine_generic_smem_kernel<l, a, b>;                                        \
            static bool attr = false;                                                               \
            if (!attr) {                                                                            \
                cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 << 10);  \
                attr = true;                                                                        \
            }                                                                                       \
            int per_sm = 1, sms = 152, dev = 0;                                                     \
            cudaGetDevice(&dev);                                                                    \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 512, smem);                 \
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);                      \
            const int64_t gs = std::min<int64_t>(rows, (int64_t)std::max(1, per_sm) * sms);         \
            kfn<<<(unsigned)gs, 512, smem, st>>>(rows, Ch, Chs, Cas, Cps, npairs, pairs, act, agg, out, k, cv, rm_h, \
                                                 elig, E);                                                       \
        } else {                                                                                    \
            combine_generic_kernel<l, a, b><<<g, 256, 0, st>>>(rows, Ch, Chs, Cas, Cps, npairs, pairs, act, agg, out, \
                                                               k, cv, rm_h, elig, E);                                 \
        }                                                                                           \
        break;
    switch ((L - 1) * 16 + (La - 1) * 4 + (Lb - 1)) {
        CC_CG(1, 1, 1)
        CC_CG(2, 1, 1) CC_CG(2, 1, 2) CC_CG(2, 2, 1) CC_CG(2, 2, 2)
        CC_CG(3, 1, 1) CC_CG(3, 1, 2) CC_CG(3, 1, 3) CC_CG(3, 2, 1) CC_CG(3, 2, 2) CC_CG(3, 2, 3)
        CC_CG(3, 3, 1) CC_CG(3, 3, 2) CC_CG(3, 3, 3)
        CC_CG(4, 1, 1) CC_CG(4, 1, 2) CC_CG(4, 1, 3) CC_CG(4, 1, 4) CC_CG(4, 2, 1) CC_CG(4, 2, 2)
        CC_CG(4, 2, 3) CC_CG(4, 2, 4) CC_CG(4, 3, 1) CC_CG(4, 3, 2) CC_CG(4, 3, 3) CC_CG(4, 3, 4)
        CC_CG(4, 4, 1) CC_CG(4, 4, 2) CC_CG(4, 4, 3) CC_CG(4, 4, 4)
    default: break;
    }
#undef CC_CG
}

}  // namespace cc
