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
// compare it with exact rational sums and dot products.
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

SSCG_HD int max_i(int a, int b) { return a > b ? a : b; }

SSCG_HD int fix_exp(uint64_t b) { return (int)((b >> 52) & 0x7FFu); }

// m >> sh for 0 <= sh; shift amounts of 64 or more give 0 (PTX clamps them).
SSCG_HD uint64_t fix_shr(uint64_t m, int sh) {
#if defined(__CUDA_ARCH__)
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(m), "r"(sh));
    return r;
#else
    return sh >= 64 ? 0ull : m >> sh;
#endif
}

// The magnitude a with the sign of the FP64 bit pattern b: (a ^ s) - s with
// s all ones for a negative b.
SSCG_HD int64_t fix_apply_sign(uint64_t a, uint64_t b) {
    const uint64_t sg = (uint64_t)((int64_t)b >> 63);
    return (int64_t)((a ^ sg) - sg);
}

// Round the value acc 2^(e0 - 1075) (|acc| < 2^63) to FP64, to nearest with
// ties to even.  Returns true with the bit pattern in *out (+0 for acc = 0),
// or false when the result is not a normal FP64 number.
SSCG_HD bool fix_pack(int64_t acc, int e0, uint64_t* out) {
    if (acc == 0) {
        *out = 0ull;  // +0, as x + (-x) gives in FP64
        return true;
    }
    const uint64_t sg = (uint64_t)(acc >> 63);
    const uint64_t mag = ((uint64_t)acc ^ sg) - sg;  // |acc| < 2^63
    const int lz = fix_clz64(mag);                   // >= 1
    const uint64_t nrm = mag << lz;                  // leading bit at bit 63
    // 53 bits rounded to nearest, ties to even: bits 63..11 plus the round bit
    // (10) when the sticky bits (9..0) or the last kept bit (11) are set
    const uint64_t keep = nrm >> 11;
    const uint64_t up = (nrm >> 10) & (keep | (uint64_t)((nrm & 0x3FFull) != 0)) & 1ull;
    const int E = e0 - lz + 11;  // biased exponent of mag 2^(e0 - 1075): leading bit 63 - lz
    if (E <= 0 || E >= 0x7FF) return false;  // a subnormal result, or overflow
    // the exponent field E - 1 plus the mantissa with its implicit bit: a
    // rounding carry into bit 53 raises the exponent by one
    const uint64_t bits = ((uint64_t)(E - 1) << 52) + keep + up;
    if ((bits >> 52) >= 0x7FF) return false;  // rounded up to overflow
    *out = bits | (sg << 63);
    return true;
}

#if defined(__CUDACC__)
// fix_pack on the conversion unit, for 53 <= e0 <= 2035 (then every nonzero
// |R| < 2^63 lands in the normal range): R rounded to FP64 (to nearest, ties
// to even) and scaled by 2^(e0 - 1075) exactly through its exponent field.
// The same result as fix_pack; the conversion runs at the FP64 rate.
__device__ __forceinline__ double fix_pack_cvt(int64_t R, int e0) {
    const double d = (double)R;
    const long long b = __double_as_longlong(d) + ((long long)(e0 - 1075) << 52);
    return R == 0 ? 0.0 : __longlong_as_double(b);
}
#endif

// Sum of the K values with raw FP64 bit patterns t[0..K-1] (K <= 31).
// Returns true with the FP64 bit pattern of the rounded sum in *out, or
// false when the fixed-point path does not apply (see the file comment).
template <int K>
SSCG_HD bool fixsum(const uint64_t (&t)[K], uint64_t* out) {
    static_assert(K >= 1 && K <= 31, "4 guard bits leave room for 31 terms below 2^57");
    int emax = 0;
#pragma unroll
    for (int k = 0; k < K; k++) emax = max_i(emax, fix_exp(t[k]));
    if (emax == 0x7FF) return false;  // a NaN or an infinity
    if (emax < 57) {                  // the result's scale 2^(emax - 1079) would not be a normal number
        uint64_t any = 0;
#pragma unroll
        for (int k = 0; k < K; k++) any |= t[k] << 1;  // nonzero unless the term is +0 or -0
        if (any) return false;
        *out = 0ull;  // every term is zero
        return true;
    }
    int64_t acc = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
        // the implicit bit is set for zeros and subnormals too: their shift emax - 0 >= 57 clears them
        const uint64_t m = ((t[k] & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 4;  // < 2^57
        acc += fix_apply_sign(fix_shr(m, emax - fix_exp(t[k])), t[k]);
    }
#if defined(__CUDA_ARCH__)
    if (emax <= 2039) {  // e0 = emax - 4 <= 2035: round on the conversion unit
        *out = (uint64_t)__double_as_longlong(fix_pack_cvt(acc, emax - 4));
        return true;
    }
#endif
    return fix_pack(acc, emax - 4, out);  // acc counts units of 2^(emax - 1079)
}

// ---------------------------------------------------------------------------
// Short dot products  v_0 c_0 + ... + v_{K-1} c_{K-1}  of FP64 values v (one
// row's entries of a few vectors) with FP64 coefficients c that are the same
// for every row (one column of a small matrix), on the integer multipliers.
// The values of a row are aligned to the row's largest exponent E and the
// coefficients of a column to the column's largest exponent Fc, both with
// kFixGuard guard bits:
//   a = trunc(v 2^(1075 + kFixGuard - E)),  C = round(c 2^(1075 + kFixGuard - Fc)),
// so |a|, |C| < 2^61 (53 significant bits and 8 guard bits).  Each is split
// into signed 32-bit limbs, a = a_h 2^32 + a_l with a_l in [-2^31, 2^31), and
// the products are summed with 32 x 32 -> 64-bit multiply-adds:
//   hh = sum a_h C_h,  ma = sum a_h C_l,  mc = sum a_l C_h   (all exact)
//   R  = hh + round(ma / 2^32) + round(mc / 2^32)
// (the a_l C_l products, below 2^62, are dropped); R 2^(E + Fc - 2102)
// approximates the dot product and is rounded once to FP64.  For K <= 7
// terms every sum stays below 2^63 (|a_h|, |C_h| <= 2^29 and |a_l|, |C_l| <=
// 2^31: each mid product below 2^60, seven of them below 2^62.9).  Error: the
// dropped products and the two roundings, at most (1 + K/4) 2^64 units of
// a C, and the truncation of a and the rounding of C, below K (2^61 + 2^60)
// units; in all at most (1 + 7K/16) 2^(E + Fc - 2102), that is
// (1 + 7K/16) 2^-56 times the row's largest |v| times the column's largest
// |c|, plus half an ulp of the result.  A sequence of K - 1 FP64 fused
// multiply-adds is bounded by (K - 1) 2^-53 sum |v c|: on vectors of similar
// magnitude the fixed-point error is the smaller of the two.
constexpr int kFixGuard = 8;
constexpr int kFixMaxTerms = 7;

struct FixLimbs {
    int32_t h, l;  // value h 2^32 + l
};

// ma and mc start at 2^31, so that their high words are the rounded
// quotients by 2^32.
struct FixAcc {
    int64_t hh = 0, ma = 0x80000000ll, mc = 0x80000000ll;
};

// a = h 2^32 + l with l the low word read as a signed number: h is the high
// word plus one when l < 0.
SSCG_HD FixLimbs fix_split(int64_t a) {
    FixLimbs r;
    const uint32_t lo = (uint32_t)(uint64_t)a;
    r.l = (int32_t)lo;
    r.h = (int32_t)((uint32_t)((uint64_t)a >> 32) + (lo >> 31));
    return r;
}

// The aligned value a = trunc(v 2^(1075 + kFixGuard - E)) of the FP64 value
// with bit pattern b, for a row exponent E >= the value's exponent and
// E >= 62 (then subnormal values, below 2^-1022, truncate to 0).
SSCG_HD FixLimbs fix_align(uint64_t b, int E) {
    // the implicit bit is set for zeros and subnormals too: with E >= 62 their
    // shift E - 0 clears them (m < 2^61)
    const uint64_t m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << kFixGuard;  // < 2^61
    return fix_split(fix_apply_sign(fix_shr(m, E - fix_exp(b)), b));
}

// The aligned coefficient C = round(c 2^(1075 + kFixGuard - Fc)) (ties away
// from zero) of the FP64 coefficient with bit pattern b, for a column
// exponent Fc >= the coefficient's exponent and Fc >= 63 (then subnormal
// coefficients round to 0).
SSCG_HD FixLimbs fix_coef(uint64_t b, int Fc) {
    const int e = fix_exp(b);
    const int d = Fc - e;
    const uint64_t m = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << kFixGuard;  // < 2^61
    int64_t c;
    if (e == 0 || d >= 63) c = 0;  // below 2^-1022, or below half a unit
    else c = (int64_t)(d == 0 ? m : ((m >> (d - 1)) + 1) >> 1);
    if (b >> 63) c = -c;
    return fix_split(c);
}

// acc += a b for signed 32-bit a, b (exact in 64 bits): one mad.wide.s32.
SSCG_HD void fix_mad_wide(int64_t& acc, int32_t a, int32_t b) {
#if defined(__CUDA_ARCH__)
    asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
#else
    acc += (int64_t)a * (int64_t)b;
#endif
}

SSCG_HD void fix_mad(FixAcc& s, FixLimbs a, FixLimbs c) {
    fix_mad_wide(s.hh, a.h, c.h);
    fix_mad_wide(s.ma, a.h, c.l);
    fix_mad_wide(s.mc, a.l, c.h);
}

// R of the accumulated products (units of 2^64 of a C).
SSCG_HD int64_t fix_total(const FixAcc& s) { return s.hh + (s.ma >> 32) + (s.mc >> 32); }

// The exponent offset e0 of a dot product: R 2^(e0 - 1075) = R 2^(E + Fc - 2102).
SSCG_HD int fix_dot_e0(int E, int Fc) { return E + Fc - 2 * kFixGuard - 1011; }

// The FP64 dot product from R, for row exponent E and column exponent Fc:
// R 2^(E + Fc - 2102) rounded to nearest; false when not a normal number.
SSCG_HD bool fix_dot_result(const FixAcc& s, int E, int Fc, uint64_t* out) {
    return fix_pack(fix_total(s), fix_dot_e0(E, Fc), out);
}



#if defined(__CUDACC__)
// Column j of the block update's coefficients [1; beta_0j .. beta_{S-1}j]
// (beta column-major, leading dimension S): returns its exponent (at least
// 1023, the exponent of the 1; 0x7FF when a coefficient is not finite) and
// stores its aligned coefficients in out.
template <int S>
__device__ __forceinline__ int fix_coef_column(const double* beta, int j, FixLimbs (&out)[S + 1]) {
    int Fc = 1023;
    for (int l = 0; l < S; l++) Fc = max_i(Fc, fix_exp((uint64_t)__double_as_longlong(beta[l + j * S])));
    out[0] = fix_coef((uint64_t)__double_as_longlong(1.0), Fc);
    for (int l = 0; l < S; l++)
        out[1 + l] = Fc < 0x7FF ? fix_coef((uint64_t)__double_as_longlong(beta[l + j * S]), Fc) : FixLimbs{0, 0};
    return Fc;
}

// The row exponents [*Elo, *Ehi] that take the fixed point with column
// exponents fc: every result offset e0 = E + Fc - 1027 in [53, 2035]
// (fix_pack_cvt) and E >= 62 (fix_align); an empty range when a coefficient
// is not finite.
template <int S>
__device__ __forceinline__ void fix_row_range(const int (&fc)[S], int* Elo, int* Ehi) {
    int fcmin = 0x7FF, fcmax = 0;
#pragma unroll
    for (int j = 0; j < S; j++) {
        fcmin = fcmin < fc[j] ? fcmin : fc[j];
        fcmax = max_i(fcmax, fc[j]);
    }
    *Elo = max_i(62, 53 - fix_dot_e0(0, fcmin));
    const int hi = 2035 - fix_dot_e0(0, fcmax);
    *Ehi = fcmax == 0x7FF ? -1 : (hi < 0x7FE ? hi : 0x7FE);
}

// One half of the fixed-point block update: out_j = v_j + sum_l w_l beta_lj
// (j < S) for one row's values v_0..v_{S-1} and w_0..w_{S-1}, all aligned to
// their largest exponent E (fixsum.cuh), the coefficient column j of [1; beta]
// in scf[j] with exponent fc[j].  Returns false, out untouched, when E lies
// outside [Elo, Ehi].
template <int S>
__device__ __forceinline__ bool fix_update_group(const double (&v)[S], const double (&w)[S],
                                                 const FixLimbs (&scf)[S][S + 1], const int (&fc)[S], int Elo,
                                                 int Ehi, double (&out)[S]) {
    unsigned hmax = 0;  // the largest exponent field (sign cleared, as an integer)
#pragma unroll
    for (int l = 0; l < S; l++)
        hmax = max(hmax, max((unsigned)__double2hiint(v[l]) & 0x7FF00000u,
                             (unsigned)__double2hiint(w[l]) & 0x7FF00000u));
    const int E = (int)(hmax >> 20);
    if (E < Elo || E > Ehi) return false;
    FixLimbs av[S], aw[S];
#pragma unroll
    for (int l = 0; l < S; l++) {
        av[l] = fix_align((uint64_t)__double_as_longlong(v[l]), E);
        aw[l] = fix_align((uint64_t)__double_as_longlong(w[l]), E);
    }
#pragma unroll
    for (int j = 0; j < S; j++) {
        FixAcc acc;
        fix_mad(acc, av[j], scf[j][0]);
#pragma unroll
        for (int l = 0; l < S; l++) fix_mad(acc, aw[l], scf[j][1 + l]);
        out[j] = fix_pack_cvt(fix_total(acc), fix_dot_e0(E, fc[j]));
    }
    return true;
}

// The same half with FP64 FMAs, in k_update_q's order.
template <int S>
__device__ __forceinline__ void fma_update_group(const double (&v)[S], const double (&w)[S], const double* sb,
                                                 double (&out)[S]) {
#pragma unroll
    for (int j = 0; j < S; j++) {
        double t = v[j];
#pragma unroll
        for (int l = 0; l < S; l++) t = ::fma(w[l], sb[l + j * S], t);
        out[j] = t;
    }
}

#endif

}  // namespace sscg
