// wideint.cuh -- fixed-width unsigned integers of L 64-bit limbs (little-endian),
// arithmetic modulo 2^(64 L).  The colour-coding DP uses only + and x, so every
// table computed modulo 2^(64 L) is the exact table reduced modulo 2^(64 L);
// a value known to be below 2^(64 L) is therefore exact.
#pragma once

#include <cstdint>

namespace cc {

template <int L>
struct Wide {
    uint64_t w[L];
};

template <int L>
__device__ __forceinline__ void wzero(Wide<L> &x)
{
#pragma unroll
    for (int i = 0; i < L; i++) x.w[i] = 0;
}

// acc += x (mod 2^(64 L))
template <int L>
__device__ __forceinline__ void wadd(Wide<L> &acc, const Wide<L> &x)
{
    if constexpr (L == 1) {
        acc.w[0] += x.w[0];
    } else {
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < L; i++) {
            uint64_t t = acc.w[i] + x.w[i];
            uint64_t c1 = t < x.w[i];
            uint64_t s = t + c;
            c1 += s < c;
            acc.w[i] = s;
            c = c1;
        }
    }
}

// acc += a * b (mod 2^(64 L)), schoolbook on limbs
template <int L>
__device__ __forceinline__ void wmac(Wide<L> &acc, const Wide<L> &a, const Wide<L> &b)
{
    if constexpr (L == 1) {
        acc.w[0] += a.w[0] * b.w[0];
    } else {
        Wide<L> p;
        wzero(p);
#pragma unroll
        for (int i = 0; i < L; i++) {
            uint64_t carry = 0;
#pragma unroll
            for (int j = 0; i + j < L; j++) {
                uint64_t lo = a.w[i] * b.w[j];
                uint64_t hi = __umul64hi(a.w[i], b.w[j]);
                uint64_t t = p.w[i + j] + lo;
                uint64_t c1 = t < lo;
                uint64_t s = t + carry;
                c1 += s < carry;
                p.w[i + j] = s;
                carry = hi + c1;
            }
        }
        wadd(acc, p);
    }
}

// acc += a * s for a small multiplier s (< 2^32 in use: colour histogram counts)
// acc += a * b mod 2^(64 L) for an La-limb a and an Lb-limb b (La, Lb <= L):
// schoolbook over the La x Lb limb products that land below limb L; the carry
// out of row i goes to limb i + Lb (still zero), or is dropped at limb L.
template <int L, int La, int Lb>
__device__ __forceinline__ void wmac_mixed(Wide<L> &acc, const Wide<La> &a, const Wide<Lb> &b)
{
    static_assert(La <= L && Lb <= L, "operands wider than the result");
    if constexpr (L == 1) {
        acc.w[0] += a.w[0] * b.w[0];
    } else {
        Wide<L> p;
        wzero(p);
#pragma unroll
        for (int i = 0; i < La; i++) {
            uint64_t carry = 0;
#pragma unroll
            for (int j = 0; j < Lb && i + j < L; j++) {
                const uint64_t lo = a.w[i] * b.w[j];
                const uint64_t hi = (i + j + 1 < L) ? __umul64hi(a.w[i], b.w[j]) : 0;
                const uint64_t t = p.w[i + j] + lo;
                uint64_t c1 = t < lo;
                const uint64_t sum = t + carry;
                c1 += sum < carry;
                p.w[i + j] = sum;
                carry = hi + c1;
            }
            if (i + Lb < L) p.w[i + Lb] = carry;
        }
        wadd(acc, p);
    }
}

template <int L>
__device__ __forceinline__ void wmac_small(Wide<L> &acc, const Wide<L> &a, uint64_t s)
{
    if constexpr (L == 1) {
        acc.w[0] += a.w[0] * s;
    } else {
        Wide<L> p;
        uint64_t carry = 0;
#pragma unroll
        for (int i = 0; i < L; i++) {
            uint64_t lo = a.w[i] * s;
            uint64_t hi = __umul64hi(a.w[i], s);
            uint64_t t = lo + carry;
            carry = hi + (t < lo);
            p.w[i] = t;
        }
        wadd(acc, p);
    }
}

// load a value stored with Ls limbs as an Ld-limb value (zero-extend or truncate)
template <int Ls, int Ld>
__device__ __forceinline__ Wide<Ld> wload(const uint64_t *__restrict__ p)
{
    Wide<Ld> r;
    if constexpr (Ls == 2 && Ld >= 2) {
        ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        r.w[0] = v.x;
        r.w[1] = v.y;
#pragma unroll
        for (int i = 2; i < Ld; i++) r.w[i] = 0;
    } else if constexpr (Ls == 4 && Ld == 4) {
        ulonglong2 v0 = __ldg(reinterpret_cast<const ulonglong2 *>(p));
        ulonglong2 v1 = __ldg(reinterpret_cast<const ulonglong2 *>(p) + 1);
        r.w[0] = v0.x; r.w[1] = v0.y; r.w[2] = v1.x; r.w[3] = v1.y;
    } else {
#pragma unroll
        for (int i = 0; i < Ld; i++) r.w[i] = (i < Ls) ? __ldg(p + i) : 0;
    }
    return r;
}

template <int L>
__device__ __forceinline__ void wstore(uint64_t *__restrict__ p, const Wide<L> &x)
{
    if constexpr (L == 2) {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x.w[0], x.w[1]);
    } else if constexpr (L == 4) {
        reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(x.w[0], x.w[1]);
        reinterpret_cast<ulonglong2 *>(p)[1] = make_ulonglong2(x.w[2], x.w[3]);
    } else {
#pragma unroll
        for (int i = 0; i < L; i++) p[i] = x.w[i];
    }
}

template <int L>
__device__ __forceinline__ Wide<L> wshfl_down(const Wide<L> &x, int d)
{
    Wide<L> r;
#pragma unroll
    for (int i = 0; i < L; i++) r.w[i] = __shfl_down_sync(0xffffffffu, x.w[i], d);
    return r;
}

}  // namespace cc
