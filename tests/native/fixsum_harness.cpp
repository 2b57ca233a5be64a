// Host build of the library's fixed-point FP64 sum, for the CPU tests
// (tests/test_fixsum_host.py): fixsum_k(k, t, out) runs fixsum<k> on the k
// bit patterns in t.
#include <stdint.h>

#include "../../paper_2501_03743_gb300/csrc/fixsum.cuh"

template <int K>
static int run(const uint64_t* t, uint64_t* out) {
    uint64_t a[K];
    for (int i = 0; i < K; i++) a[i] = t[i];
    return sscg::fixsum<K>(a, out) ? 1 : 0;
}

extern "C" int fixsum_k(int k, const uint64_t* t, uint64_t* out) {
    switch (k) {
        case 1: return run<1>(t, out);
        case 6: return run<6>(t, out);
        case 26: return run<26>(t, out);
        case 31: return run<31>(t, out);
        default: return -1;
    }
}

// fixdot_k(k, v, c, E, Fc, out): the fixed-point dot product of fixsum.cuh
// of the k values v (bit patterns) and coefficients c, with row exponent E
// and column exponent Fc; returns 1 with the FP64 bit pattern in *out, or 0.
extern "C" int fixdot_k(int k, const uint64_t* v, const uint64_t* c, int E, int Fc, uint64_t* out) {
    if (k < 1 || k > sscg::kFixMaxTerms) return -1;
    sscg::FixAcc acc;
    for (int t = 0; t < k; t++) sscg::fix_mad(acc, sscg::fix_align(v[t], E), sscg::fix_coef(c[t], Fc));
    return sscg::fix_dot_result(acc, E, Fc, out) ? 1 : 0;
}

// The aligned value and coefficient as 64-bit integers (limbs recombined).
extern "C" int64_t fix_align_value(uint64_t v, int E) {
    const sscg::FixLimbs a = sscg::fix_align(v, E);
    return (int64_t)a.h * 4294967296ll + a.l;
}

extern "C" int64_t fix_coef_value(uint64_t c, int Fc) {
    const sscg::FixLimbs a = sscg::fix_coef(c, Fc);
    return (int64_t)a.h * 4294967296ll + a.l;
}

// fix_pack_value(acc, e0, out): acc 2^(e0 - 1075) rounded to FP64 by fix_pack.
extern "C" int fix_pack_value(int64_t acc, int e0, uint64_t* out) { return sscg::fix_pack(acc, e0, out) ? 1 : 0; }
