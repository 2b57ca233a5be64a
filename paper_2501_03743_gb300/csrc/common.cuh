// Device-side building blocks shared by the sscg kernels: double-float
// arithmetic, arithmetic traits, the solver control block and deterministic
// block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sscg {

constexpr int kMaxS = 16;       // largest supported block size s
constexpr int kThreads = 256;   // threads per CTA of every row-parallel kernel
constexpr int kTileRows = 256;  // rows per SpMV tile (one per thread)

// ------------------------------------------------------------ double-float
//
// A df64 value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits.  The operations below are
// the error-free transformations TwoSum (Knuth), FastTwoSum (Dekker) and the
// FMA form of TwoProduct, and the accurate double-double addition and
// multiplication built from them (Hida, Li and Bailey, "Algorithms for
// quad-double precision floating point arithmetic", ARITH 2001).  Every
// primitive uses an explicitly rounded intrinsic so the compiler cannot
// contract or reassociate the compensation terms.

struct df64 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_make(float hi, float lo) {
    df64 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
    float s1, s2, t1, t2;
    two_sum(a.hi, b.hi, s1, s2);
    two_sum(a.lo, b.lo, t1, t2);
    s2 = __fadd_rn(s2, t1);
    fast_two_sum(s1, s2, s1, s2);
    s2 = __fadd_rn(s2, t2);
    fast_two_sum(s1, s2, s1, s2);
    return df_make(s1, s2);
}

__device__ __forceinline__ df64 df_neg(df64 a) { return df_make(-a.hi, -a.lo); }

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    fast_two_sum(p, e, s, t);
    return df_make(s, t);
}

// a * b with b an exact FP32 number.
__device__ __forceinline__ df64 df_mul_f(df64 a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    float s, t;
    fast_two_sum(p, e, s, t);
    return df_make(s, t);
}

// c + a * b: the exact product hi*hi as p + e (FMA TwoProduct) with the
// cross terms folded into e, added to c by TwoSum on the high parts and one
// renormalisation (the "sloppy" double-double addition of Hida, Li and
// Bailey): 15 FP32 operations instead of 27 for df_add(df_mul(a, b), c).
// The error is about 2^-47 of max(|c|, |a b|).
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    fast_two_sum(s, t, s, t);
    return df_make(s, t);
}

// c + a * v for an FP32 number v.
__device__ __forceinline__ df64 df_fma_f(df64 a, float v, df64 c) {
    float p = __fmul_rn(a.hi, v);
    float e = __fmaf_rn(a.hi, v, -p);
    e = __fmaf_rn(a.lo, v, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    fast_two_sum(s, t, s, t);
    return df_make(s, t);
}

__device__ __forceinline__ df64 df_from_double(double x) {
    float hi = __double2float_rn(x);
    float lo = __double2float_rn(x - (double)hi);
    return df_make(hi, lo);
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// Running double-float dot product in the cascaded form of Dot2 (Ogita, Rump
// and Oishi, "Accurate sum and dot product", 2005): the high parts of the
// products are added by TwoSum into s, every rounding error and the low-order
// product terms into e.  dot_renorm folds e back into s (FastTwoSum); called
// every couple of terms it keeps the accumulated error at the level of a
// renormalised double-float sum while a term costs 12 FP32 operations instead
// of 15.
struct DotAcc {
    float s, e;
};

__device__ __forceinline__ void dot_add(DotAcc& a, df64 x, df64 y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float q = __fmaf_rn(x.hi, y.hi, -p);
    q = __fmaf_rn(x.hi, y.lo, q);
    q = __fmaf_rn(x.lo, y.hi, q);
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, q));
}

// a += y * y (the cross term 2 y.hi y.lo with the exact doubling of y.hi)
__device__ __forceinline__ void dot_add_sq(DotAcc& a, df64 y) {
    const float p = __fmul_rn(y.hi, y.hi);
    float q = __fmaf_rn(y.hi, y.hi, -p);
    q = __fmaf_rn(__fadd_rn(y.hi, y.hi), y.lo, q);
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, q));
}

__device__ __forceinline__ void dot_renorm(DotAcc& a) {
    float s, t;
    fast_two_sum(a.s, a.e, s, t);
    a.s = s;
    a.e = t;
}

// Two consecutive double-float elements p[0], p[1] in one 16-byte store
// (p 16-byte aligned).
__device__ __forceinline__ void st_pair(float2* p, df64 a, df64 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.hi, a.lo, b.hi, b.lo);
}

__device__ __forceinline__ df64 dot_value(DotAcc a) {
    dot_renorm(a);
    return df_make(a.s, a.e);
}

// ------------------------------------------------------- arithmetic traits
//
// R: register type.  S: storage type of vectors and basis blocks.
// fma(a, b, c) = a * b + c.

struct ArithF64 {
    using R = double;
    using S = double;
    static constexpr int kind = 0;
    __device__ static __forceinline__ R zero() { return 0.0; }
    __device__ static __forceinline__ R ld(const S* p) { return *p; }
    __device__ static __forceinline__ R ldg(const S* p) { return __ldg(p); }
    __device__ static __forceinline__ R ldcg(const S* p) { return __ldcg(p); }
    __device__ static __forceinline__ void st(S* p, R v) { *p = v; }
    __device__ static __forceinline__ void st_stream(S* p, R v) { __stcs(p, v); }
    __device__ static __forceinline__ R add(R a, R b) { return a + b; }
    __device__ static __forceinline__ R sub(R a, R b) { return a - b; }
    __device__ static __forceinline__ R mul(R a, R b) { return a * b; }
    __device__ static __forceinline__ R fma(R a, R b, R c) { return ::fma(a, b, c); }
    __device__ static __forceinline__ R from_d(double x) { return x; }
    __device__ static __forceinline__ double to_d(R a) { return a; }
    __device__ static __forceinline__ R shfl_xor(R a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
};

struct ArithDF64 {
    using R = df64;
    using S = float2;
    static constexpr int kind = 1;
    __device__ static __forceinline__ R zero() { return df_make(0.f, 0.f); }
    __device__ static __forceinline__ R ld(const S* p) {
        float2 v = *p;
        return df_make(v.x, v.y);
    }
    __device__ static __forceinline__ R ldg(const S* p) {
        float2 v = __ldg(p);
        return df_make(v.x, v.y);
    }
    __device__ static __forceinline__ R ldcg(const S* p) {
        float2 v = __ldcg(p);
        return df_make(v.x, v.y);
    }
    __device__ static __forceinline__ void st(S* p, R v) { *p = make_float2(v.hi, v.lo); }
    __device__ static __forceinline__ void st_stream(S* p, R v) { __stcs(p, make_float2(v.hi, v.lo)); }
    __device__ static __forceinline__ R add(R a, R b) { return df_add(a, b); }
    __device__ static __forceinline__ R sub(R a, R b) { return df_add(a, df_neg(b)); }
    __device__ static __forceinline__ R mul(R a, R b) { return df_mul(a, b); }
    __device__ static __forceinline__ R fma(R a, R b, R c) { return df_fma(a, b, c); }
    __device__ static __forceinline__ R from_d(double x) { return df_from_double(x); }
    __device__ static __forceinline__ double to_d(R a) { return df_to_double(a); }
    __device__ static __forceinline__ R shfl_xor(R a, int m) {
        return df_make(__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m));
    }
};

// FP32 arithmetic and storage (basis blocks of the mixed-precision mode).
struct ArithF32 {
    using R = float;
    using S = float;
    static constexpr int kind = 2;
    __device__ static __forceinline__ R zero() { return 0.f; }
    __device__ static __forceinline__ R ld(const S* p) { return *p; }
    __device__ static __forceinline__ R ldg(const S* p) { return __ldg(p); }
    __device__ static __forceinline__ R ldcg(const S* p) { return __ldcg(p); }
    __device__ static __forceinline__ void st(S* p, R v) { *p = v; }
    __device__ static __forceinline__ R add(R a, R b) { return a + b; }
    __device__ static __forceinline__ R sub(R a, R b) { return a - b; }
    __device__ static __forceinline__ R mul(R a, R b) { return a * b; }
    __device__ static __forceinline__ R fma(R a, R b, R c) { return fmaf(a, b, c); }
    __device__ static __forceinline__ R from_d(double x) { return (float)x; }
    __device__ static __forceinline__ double to_d(R a) { return (double)a; }
    __device__ static __forceinline__ R shfl_xor(R a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
};

// FP32 storage with double-float accumulation: Gram sums of FP32 blocks,
// where every product of two FP32 numbers is formed exactly.
struct ArithF32Acc {
    using R = df64;
    using S = float;
    static constexpr int kind = 3;
    __device__ static __forceinline__ R zero() { return df_make(0.f, 0.f); }
    __device__ static __forceinline__ R ld(const S* p) { return df_make(*p, 0.f); }
    __device__ static __forceinline__ void st(S* p, R v) { *p = v.hi; }
    __device__ static __forceinline__ R add(R a, R b) { return df_add(a, b); }
    __device__ static __forceinline__ R fma(R a, R b, R c) { return df_fma(a, b, c); }
    __device__ static __forceinline__ R from_d(double x) { return df_from_double(x); }
    __device__ static __forceinline__ double to_d(R a) { return df_to_double(a); }
    __device__ static __forceinline__ R shfl_xor(R a, int m) {
        return df_make(__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m));
    }
};

// --------------------------------------------------------- control block
//
// One per solve, in the caller's workspace.  Kernels read `done` at entry
// and return at once when it is set, so launches queued after convergence
// or breakdown cost only their launch.

struct Ctrl {
    int done;        // nonzero: stop
    int status;      // sscg_status of the solve
    int step;        // outer steps (PCG: iterations) completed
    int maxit;
    unsigned ticket[4];  // last-CTA counters (one per kernel family)
    int s;
    int zero_rhs;    // b = 0: x is set to 0 at the end
    int nhist;       // history entries written
    int pad0;
    double tol;
    double bnorm;    // ||b||_2
    double relres;   // recursive ||r||/||b|| after the last step
    double true_res2;
    double mu[2 * kMaxS + 2];     // moments mu_0 .. mu_{2s-1}
    double W[kMaxS * kMaxS];      // column-major, current W_i
    double alpha[kMaxS];
    double beta[kMaxS * kMaxS];   // column-major
    double G[kMaxS * kMaxS];      // direct Gram blocks (Chebyshev basis)
    double C[kMaxS * kMaxS];
    double m[kMaxS];
    double q[kMaxS];              // P_old^T r (residual-replacement correction of m)
    int with_q;                   // q was formed this step
    int pad2;
    double basis_c, basis_delta;  // Chebyshev basis centre and half-width
    double rho, pcg_alpha, pcg_beta;  // PCG scalars
    double scratch[8];
    unsigned claim;  // work-item counter of the fused matrix-powers kernel
    unsigned pad1[3];
    double Wl[kMaxS * kMaxS];  // Cholesky factor of W (lower triangle), for the next step's solve
    double Wr[kMaxS];          // reciprocals of its diagonal
};

// ------------------------------------------------------------- reductions

template <class A>
__device__ __forceinline__ typename A::R warp_sum(typename A::R v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = A::add(v, A::shfl_xor(v, m));
    return v;
}

// Sum NV values over the CTA (blockDim.x a multiple of 32); the result is
// returned as doubles in thread 0.  `sh` holds NV * (blockDim.x/32) doubles.
template <class A, int NV>
__device__ __forceinline__ void block_sum(typename A::R (&v)[NV], double* sh, double (&out)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        typename A::R w = warp_sum<A>(v[q]);
        if (lane == 0) sh[q * nw + warp] = A::to_d(w);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double t = 0.0;
            for (int w = 0; w < nw; w++) t += sh[q * nw + w];
            out[q] = t;
        }
    }
    __syncthreads();
}

// Last-CTA election: every CTA calls this after writing its partials; it
// returns true in exactly one CTA (the last to arrive), in all its threads,
// after which that CTA may read every CTA's partials.  The counter is reset
// for the next launch.
__device__ __forceinline__ bool last_cta(unsigned* ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *ticket = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Deterministic sum of `count` values spaced `stride` apart, by one CTA;
// the result is valid in thread 0.  Reads bypass L1.
__device__ __forceinline__ double cta_sum_partials(const double* p, int count, double* sh) {
    double t = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) t += __ldcg(p + i);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = t;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); w++) r += sh[w];
    __syncthreads();
    return r;
}

// Maximum of v over the CTA, valid in thread 0 (blockDim.x a multiple of 32;
// `sh` holds blockDim.x / 32 doubles).  Ends with a CTA barrier.
__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / 32); w++) r = fmax(r, sh[w]);
    __syncthreads();
    return r;
}

// Maximum of `count` nonnegative values, by one CTA; valid in thread 0.
__device__ __forceinline__ double cta_max_partials(const double* p, int count, double* sh) {
    double t = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) t = fmax(t, __ldcg(p + i));
    __syncthreads();
    return block_max(t, sh);
}

// Right-hand sides a double-float or mixed solve accepts: max |b_i| in
// [2^-30, 2^30].  Their vectors, squared norms and moments live in FP32's
// exponent range (about 1e-38 ... 3e38); a right-hand side far outside O(1)
// would underflow or overflow them before the solve reached its tolerance.
constexpr double kDfRhsMin = 0x1p-30, kDfRhsMax = 0x1p30;

// Deterministic sums of `count` partial arrays (array e holds G values at
// p + e*G) by one CTA, warps taking arrays round-robin; store(e, value) runs
// in lane 0 of the owning warp.  Ends with a CTA barrier.
template <class F>
__device__ __forceinline__ void cta_sum_rows(const double* p, int count, int G, F store) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = warp; e < count; e += nw) {
        double t = 0.0;
        for (int i = lane; i < G; i += 32) t += __ldcg(p + (size_t)e * G + i);
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
        if (lane == 0) store(e, t);
    }
    __syncthreads();
}

}  // namespace sscg
