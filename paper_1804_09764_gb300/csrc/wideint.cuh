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

// acc += x (mod 2^(64 L)): one add-with-carry chain over the limbs
template <int L>
__device__ __forceinline__ void wadd(Wide<L> &acc, const Wide<L> &x)
{
    if constexpr (L == 1) {
        acc.w[0] += x.w[0];
    } else if constexpr (L == 2) {
        asm("add.cc.u64 %0, %0, %2;\n\t"
            "addc.u64 %1, %1, %3;"
            : "+l"(acc.w[0]), "+l"(acc.w[1])
            : "l"(x.w[0]), "l"(x.w[1]));
    } else if constexpr (L == 3) {
        asm("add.cc.u64 %0, %0, %3;\n\t"
            "addc.cc.u64 %1, %1, %4;\n\t"
            "addc.u64 %2, %2, %5;"
            : "+l"(acc.w[0]), "+l"(acc.w[1]), "+l"(acc.w[2])
            : "l"(x.w[0]), "l"(x.w[1]), "l"(x.w[2]));
    } else {
        static_assert(L == 4, "1 to 4 limbs");
        asm("add.cc.u64 %0, %0, %4;\n\t"
            "addc.cc.u64 %1, %1, %5;\n\t"
            "addc.cc.u64 %2, %2, %6;\n\t"
            "addc.u64 %3, %3, %7;"
            : "+l"(acc.w[0]), "+l"(acc.w[1]), "+l"(acc.w[2]), "+l"(acc.w[3])
            : "l"(x.w[0]), "l"(x.w[1]), "l"(x.w[2]), "l"(x.w[3]));
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

// acc += a * s (mod 2^(64 L)) for a one-limb multiplier s (in use: colour
// histogram counts)
template <int L>
__device__ __forceinline__ void wmac_small(Wide<L> &acc, const Wide<L> &a, uint64_t s)
{
    // the low halves of a_i * s go into limb i, the high halves into limb i + 1:
    // two add-with-carry chains of multiply-adds
    if constexpr (L == 1) {
        acc.w[0] += a.w[0] * s;
    } else if constexpr (L == 2) {
        asm("mad.lo.cc.u64 %0, %2, %4, %0;\n\t"
            "madc.lo.u64 %1, %3, %4, %1;\n\t"
            "mad.hi.u64 %1, %2, %4, %1;"
            : "+l"(acc.w[0]), "+l"(acc.w[1])
            : "l"(a.w[0]), "l"(a.w[1]), "l"(s));
    } else if constexpr (L == 3) {
        asm("mad.lo.cc.u64 %0, %3, %6, %0;\n\t"
            "madc.lo.cc.u64 %1, %4, %6, %1;\n\t"
            "madc.lo.u64 %2, %5, %6, %2;\n\t"
            "mad.hi.cc.u64 %1, %3, %6, %1;\n\t"
            "madc.hi.u64 %2, %4, %6, %2;"
            : "+l"(acc.w[0]), "+l"(acc.w[1]), "+l"(acc.w[2])
            : "l"(a.w[0]), "l"(a.w[1]), "l"(a.w[2]), "l"(s));
    } else {
        static_assert(L == 4, "1 to 4 limbs");
        asm("mad.lo.cc.u64 %0, %4, %8, %0;\n\t"
            "madc.lo.cc.u64 %1, %5, %8, %1;\n\t"
            "madc.lo.cc.u64 %2, %6, %8, %2;\n\t"
            "madc.lo.u64 %3, %7, %8, %3;\n\t"
            "mad.hi.cc.u64 %1, %4, %8, %1;\n\t"
            "madc.hi.cc.u64 %2, %5, %8, %2;\n\t"
            "madc.hi.u64 %3, %6, %8, %3;"
            : "+l"(acc.w[0]), "+l"(acc.w[1]), "+l"(acc.w[2]), "+l"(acc.w[3])
            : "l"(a.w[0]), "l"(a.w[1]), "l"(a.w[2]), "l"(a.w[3]), "l"(s));
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

// Running sum of neighbour values stored with Ls limbs, for an Ld-limb result.
// The low N = min(Ls, Ld) limbs are summed with one add-with-carry chain; when
// Ld > Ls the carries out of limb Ls - 1 go to a 32-bit counter instead of
// full limbs: a sum of at most 2^31 values (a CSR neighbour list is shorter
// than that) below 2^(64 Ls) is below 2^31 * 2^(64 Ls), so limb Ls of the sum
// is that count and every limb above it is zero.  When Ld <= Ls the sum is
// taken modulo 2^(64 Ld) on the low Ld limbs of each value.
template <int Ls, int Ld>
struct RowSum {
    static constexpr int N = Ls < Ld ? Ls : Ld;
    static constexpr bool kCarry = Ld > Ls;
    Wide<N> s;   // the low N limbs
    uint32_t c;  // carries out of limb N - 1 (kCarry only)

    __device__ __forceinline__ void zero()
    {
        wzero(s);
        c = 0;
    }
    // the low N limbs of the value at p (Ls limbs; 16-byte aligned when Ls is even)
    __device__ __forceinline__ static Wide<N> load(const uint64_t *__restrict__ p)
    {
        Wide<N> r;
        if constexpr (N == 2 && Ls % 2 == 0) {
            const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
            r.w[0] = v.x;
            r.w[1] = v.y;
        } else if constexpr (N == 4) {
            const ulonglong2 v0 = __ldg(reinterpret_cast<const ulonglong2 *>(p));
            const ulonglong2 v1 = __ldg(reinterpret_cast<const ulonglong2 *>(p) + 1);
            r.w[0] = v0.x; r.w[1] = v0.y; r.w[2] = v1.x; r.w[3] = v1.y;
        } else {
#pragma unroll
            for (int i = 0; i < N; i++) r.w[i] = __ldg(p + i);
        }
        return r;
    }
    __device__ __forceinline__ void add(const Wide<N> &x)
    {
        if constexpr (!kCarry) {
            wadd(s, x);
        } else if constexpr (N == 1) {
            asm("add.cc.u64 %0, %0, %2;\n\t"
                "addc.u32 %1, %1, 0;"
                : "+l"(s.w[0]), "+r"(c)
                : "l"(x.w[0]));
        } else if constexpr (N == 2) {
            asm("add.cc.u64 %0, %0, %3;\n\t"
                "addc.cc.u64 %1, %1, %4;\n\t"
                "addc.u32 %2, %2, 0;"
                : "+l"(s.w[0]), "+l"(s.w[1]), "+r"(c)
                : "l"(x.w[0]), "l"(x.w[1]));
        } else {
            static_assert(N == 3, "a carry counter needs Ls < Ld <= 4");
            asm("add.cc.u64 %0, %0, %4;\n\t"
                "addc.cc.u64 %1, %1, %5;\n\t"
                "addc.cc.u64 %2, %2, %6;\n\t"
                "addc.u32 %3, %3, 0;"
                : "+l"(s.w[0]), "+l"(s.w[1]), "+l"(s.w[2]), "+r"(c)
                : "l"(x.w[0]), "l"(x.w[1]), "l"(x.w[2]));
        }
    }
    __device__ __forceinline__ Wide<Ld> wide() const
    {
        Wide<Ld> r;
#pragma unroll
        for (int i = 0; i < Ld; i++) r.w[i] = i < N ? s.w[i] : (kCarry && i == N ? (uint64_t)c : 0);
        return r;
    }
};

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
