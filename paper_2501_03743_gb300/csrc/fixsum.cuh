// Sums of a few FP64 values on the integer units.
//
// On a GB300 the FP64 units retire about 2 operations per clock per SM and
// the integer units about 80, so a stencil row's neighbour sum (5 FP64
// additions for the 7-point stencil, 25 for the 27-point one) is cheaper in
// 64-bit fixed point: every term's 53-bit significand is aligned to the
// largest term's exponent with 4 guard bits (a right shift, the bits shifted
// out dropped), the aligned terms are added as two's-complement integers
// (exact: at most 31 terms of less than 2^57 each), and the integer sum is
// rounded once to FP64 (round to nearest, ties to even).  The error is at
// most K 2^(e_max - 1079) from the dropped bits (K terms, e_max the largest
// biased exponent: K 2^-56 of the largest term's magnitude) plus half an ulp
// of the result, inside the (K - 1) 2^-53 sum|term| bound of K - 1 FP64
// additions in sequence.  Terms that are NaN or infinite, rows whose largest
// term is below 2^-966, and results outside the normal range take no fixed-
// point path: fixsum returns false and the caller adds in FP64 (a row of
// zeros sums to +0).
//
// Integer code only (host and device), so the CPU tests compile it and
// compare it with exact rational sums.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define SSCG_HD __host__ __device__ __forceinline__
#else
#define SSCG_HD inline
#endif

namespace sscg {

SSCG_HD int fix_clz64(uint64_t v) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return __builtin_clzll(v);
#endif
}

// Sum of the K values with raw FP64 bit patterns t[0..K-1] (K <= 31).
// Returns true with the FP64 bit pattern of the rounded sum in *out, or
// false when the fixed-point path does not apply (see the file comment).
template <int K>
SSCG_HD bool fixsum(const uint64_t (&t)[K], uint64_t* out) {
    static_assert(K >= 1 && K <= 31, "4 guard bits leave room for 31 terms below 2^57");
    int emax = 1;
    uint64_t any = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int E = (int)((t[k] >> 52) & 0x7FFu);
        if (E == 0x7FF) return false;  // NaN or infinity
        emax = E > emax ? E : emax;    // subnormals (E = 0) share exponent 1 without the implicit bit
        any |= t[k] << 1;              // nonzero unless the term is +0 or -0
    }
    if (emax < 57) {  // the result's scale 2^(emax - 1079) would not be a normal number
        if (any) return false;
        *out = 0ull;  // every term is zero
        return true;
    }
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int E = (int)((t[k] >> 52) & 0x7FFu);
        const uint64_t implicit = E ? (1ull << 52) : 0ull;
        const uint64_t m = ((t[k] & 0xFFFFFFFFFFFFFull) | implicit) << 4;  // < 2^57
        const int sh = emax - (E ? E : 1);
        const int64_t a = sh >= 64 ? 0 : (int64_t)(m >> sh);
        acc += (t[k] >> 63) ? -a : a;
    }
    if (acc == 0) {
        *out = 0ull;  // +0, as x + (-x) gives in FP64
        return true;
    }
    const uint64_t sign = acc < 0 ? (1ull << 63) : 0ull;
    uint64_t mag = acc < 0 ? (uint64_t)(-acc) : (uint64_t)acc;  // < 2^62
    const int p = 63 - fix_clz64(mag);                          // leading bit: mag in [2^p, 2^(p+1))
    int E = p + emax - 56;                                      // biased exponent of mag 2^(emax - 1079)
    uint64_t mant;
    if (p <= 52) {
        mant = mag << (52 - p);  // exact
    } else {
        const int sh = p - 52;
        mant = mag >> sh;
        const uint64_t rem = mag & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) mant++;
        if (mant == (1ull << 53)) {  // rounding carried into a new leading bit
            mant >>= 1;
            E++;
        }
    }
    if (E >= 0x7FF) return false;  // overflow: the FP64 additions give the infinity
    *out = sign | ((uint64_t)E << 52) | (mant & 0xFFFFFFFFFFFFFull);
    return true;
}

}  // namespace sscg
