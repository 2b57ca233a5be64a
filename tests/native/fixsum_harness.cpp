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
