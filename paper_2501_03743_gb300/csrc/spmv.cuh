// CSR row-tile SpMV shared by every kernel that multiplies by A.
//
// A CTA takes a tile of kTileRows consecutive rows.  It loads the tile's
// row pointers, then copies the tile's contiguous column-index and value
// ranges into shared memory with coalesced loads, and each thread forms the
// dot product of one row from shared memory, gathering x[col] through the
// read-only cache.  Tiles whose entries exceed the staging capacity take the
// remainder straight from global memory.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fixsum.cuh"
#include "internal.h"

namespace sscg {

// How the matrix values are stored and multiplied.
enum ValMode { VAL_F64 = 0, VAL_F32 = 1, VAL_DF = 2 };

constexpr int kDiaMax = 32;

struct MatView {
    int n;
    int cap;  // staging capacity (entries) of the dynamic shared memory
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
    const float* __restrict__ vhi;
    const float* __restrict__ vlo;
    // constant-coefficient diagonal form (used when the kernel is built for it)
    const uint32_t* __restrict__ dmask;
    int dk;
    int doff[kDiaMax];
    double dc[kDiaMax];
    int dcen;   // index of offset 0
    int dlap;   // every off-centre coefficient equals dco
    float dco;  // that coefficient
    int deven;  // every offset beyond the centre's two sorted neighbours is even
};

// The kernels' view of a matrix: its CSR arrays and, when it has one, its
// constant-coefficient diagonal form.
inline MatView mat_view(const sscg_mat* m) {
    MatView v{};
    v.n = (int)m->n;
    v.cap = stage_cap(m);
    v.rowptr = m->rowptr;
    v.col = m->col;
    v.val = m->val;
    v.vhi = m->vhi;
    v.vlo = m->vlo;
    v.dmask = m->dia_mask;
    v.dk = m->dia ? m->dia_k : 0;
    for (int t = 0; t < kDiaMax; t++) {
        v.doff[t] = t < v.dk ? m->dia_off[t] : 0;
        v.dc[t] = t < v.dk ? m->dia_c[t] : 0.0;
    }
    v.dcen = m->dia_cen;
    v.dlap = m->dia_lap;
    v.dco = (float)m->dia_co;
    v.deven = 1;
    for (int t = 0; t < v.dk; t++)
        if ((t < m->dia_cen - 1 || t > m->dia_cen + 1) && (v.doff[t] & 1)) v.deven = 0;
    return v;
}

template <class A, int VM>
struct Val;

template <>
struct Val<ArithF64, VAL_F64> {
    using T = double;
    __device__ static __forceinline__ T load(const MatView& M, int k) { return __ldg(M.val + k); }
    __device__ static __forceinline__ double mac(double acc, T v, double x) { return ::fma(v, x, acc); }
};

template <>
struct Val<ArithDF64, VAL_F32> {
    using T = float;
    __device__ static __forceinline__ T load(const MatView& M, int k) { return __ldg(M.vhi + k); }
    __device__ static __forceinline__ df64 mac(df64 acc, T v, df64 x) { return df_fma_f(x, v, acc); }
};

template <>
struct Val<ArithF32, VAL_F32> {
    using T = float;
    __device__ static __forceinline__ T load(const MatView& M, int k) { return __ldg(M.vhi + k); }
    __device__ static __forceinline__ float mac(float acc, T v, float x) { return fmaf(v, x, acc); }
};

template <>
struct Val<ArithDF64, VAL_DF> {
    using T = float2;
    __device__ static __forceinline__ T load(const MatView& M, int k) {
        return make_float2(__ldg(M.vhi + k), __ldg(M.vlo + k));
    }
    __device__ static __forceinline__ df64 mac(df64 acc, T v, df64 x) { return df_fma(x, df_make(v.x, v.y), acc); }
};

// Bytes of dynamic shared memory for a staging capacity of `cap` entries.
template <class A, int VM>
__host__ __device__ constexpr size_t stage_bytes(int cap) {
    return ((size_t)cap * 4 + 15) / 16 * 16 + (size_t)cap * sizeof(typename Val<A, VM>::T);
}

// y = (A x)[row] for the calling thread's row of `tile`; every thread of the
// CTA must call it (it synchronises).  Returns false for threads past the
// last row.  `xf(c)` loads x[c] as A::R.
template <class A, int VM, class XF>
__device__ __forceinline__ bool tile_spmv(const MatView& M, int tile, XF xf, typename A::R& y, int& row,
                                          char* smem, int* s_rp) {
    using V = Val<A, VM>;
    using T = typename V::T;
    const int r0 = tile * kTileRows;
    const int nrows = min(kTileRows, M.n - r0);
    __syncthreads();  // previous tile is done with the staging buffers
    for (int t = threadIdx.x; t <= nrows; t += blockDim.x) s_rp[t] = __ldg(M.rowptr + r0 + t);
    __syncthreads();
    const int base = s_rp[0];
    const int cnt = s_rp[nrows] - base;
    const int staged = min(cnt, M.cap);
    int32_t* s_col = (int32_t*)smem;
    T* s_val = (T*)(smem + ((size_t)M.cap * 4 + 15) / 16 * 16);
    for (int k = threadIdx.x; k < staged; k += blockDim.x) {
        s_col[k] = __ldg(M.col + base + k);
        s_val[k] = V::load(M, base + k);
    }
    __syncthreads();
    row = r0 + threadIdx.x;
    y = A::zero();
    if (threadIdx.x >= nrows) return false;
    const int ks = s_rp[threadIdx.x] - base, ke = s_rp[threadIdx.x + 1] - base;
    const int km = min(ke, staged);
    for (int k = ks; k < km; k++) y = V::mac(y, s_val[k], xf(s_col[k]));
    for (int k = max(ks, staged); k < ke; k++) y = V::mac(y, V::load(M, base + k), xf(__ldg(M.col + base + k)));
    return true;
}

// y = (A x)[i] for every row i of a matrix in constant-coefficient diagonal
// form: y_i = sum over the offsets t that row i holds of c_t x[i + off_t].
// No column indices or values are read: one 32-bit presence mask per row.
// Rows are taken grid-stride, so a warp gathers 32 consecutive x entries per
// offset.  `epi(row, y)` consumes each result.  Every thread must call it.
//
// In double-float the row sum is a cascaded dot product (Dot2 of Ogita,
// Rump and Oishi, "Accurate sum and dot product", 2005): each c_t x_t is
// split exactly into p + e (FMA TwoProduct of c_t and x_t.hi, plus c_t x_t.lo
// folded into e), the p are added by TwoSum into one float, every rounding
// error and e into a second float, and the pair is renormalised once per
// row: 11 FP32 operations per entry instead of 14 for a renormalised
// double-float multiply-add each.
struct Dot2Acc {
    float s, e;
};

__device__ __forceinline__ void dot2_add(Dot2Acc& a, float c, df64 x) {
    const float p = __fmul_rn(c, x.hi);
    float q = __fmaf_rn(c, x.hi, -p);
    q = __fmaf_rn(c, x.lo, q);
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, q));
}

// The same for a coefficient that is a power of two (the stencils' -1):
// c x.hi and c x.lo are exact, so no TwoProduct is needed.
__device__ __forceinline__ void dot2_add_pow2(Dot2Acc& a, float c, df64 x) {
    const float p = __fmul_rn(c, x.hi);
    const float q = __fmul_rn(c, x.lo);
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, q));
}

__host__ __device__ inline bool is_pow2_float(float c) {
    if (!(c != 0.0f)) return false;
    const float a = c < 0.f ? -c : c;
    int e = 0;
    return frexpf(a, &e) == 0.5f;
}

__device__ __forceinline__ df64 dot2_result(const Dot2Acc& a) {
    float s, t;
    fast_two_sum(a.s, a.e, s, t);
    return df_make(s, t);
}

template <class A, int KM, class XF, class EPI>
__device__ __forceinline__ void spmv_dia_rows(const MatView& M, const int* s_off, const double* s_c,
                                              const float* s_cf, XF xf, EPI epi) {
    using R = typename A::R;
    const int K = M.dk;
    const int last = M.n - 1;
    // up to 8 offsets: offsets and coefficients in registers
    int off[KM <= 8 ? KM : 1];
    float cf[KM <= 8 ? KM : 1];
    double cd[KM <= 8 ? KM : 1];
    bool p2[KM <= 8 ? KM : 1];
    if constexpr (KM <= 8) {
#pragma unroll
        for (int t = 0; t < KM; t++) {
            off[t] = t < K ? s_off[t] : 0;
            cf[t] = t < K ? s_cf[t] : 0.f;
            cd[t] = t < K ? s_c[t] : 0.0;
            p2[t] = is_pow2_float(cf[t]);
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M.n; i += gridDim.x * blockDim.x) {
        // The gathers do not wait for the mask: every offset is loaded at an
        // index clamped into [0, n), and the mask only selects which terms
        // enter the sum, so the loads issue together with the mask's.
        const uint32_t m = __ldg(M.dmask + i);
        if constexpr (KM <= 8) {
            R xv[KM];
#pragma unroll
            for (int t = 0; t < KM; t++)
                if (t < K) xv[t] = xf(min(max(i + off[t], 0), last));
            if constexpr (A::kind == 0) {
                double y = 0.0;
#pragma unroll
                for (int t = 0; t < KM; t++)
                    if (t < K && ((m >> t) & 1u)) y = ::fma(cd[t], xv[t], y);
                epi(i, y);
            } else {
                Dot2Acc acc{0.f, 0.f};
#pragma unroll
                for (int t = 0; t < KM; t++)
                    if (t < K && ((m >> t) & 1u)) {
                        if (p2[t]) dot2_add_pow2(acc, cf[t], xv[t]);  // uniform: same offset for every row
                        else dot2_add(acc, cf[t], xv[t]);
                    }
                epi(i, R(dot2_result(acc)));
            }
        } else {
            if constexpr (A::kind == 0) {
                double y = 0.0;
                for (int t = 0; t < K; t++)
                    if ((m >> t) & 1u) y = ::fma(s_c[t], xf(i + s_off[t]), y);
                epi(i, y);
            } else {
                Dot2Acc acc{0.f, 0.f};
                for (int t = 0; t < K; t++)
                    if ((m >> t) & 1u) dot2_add(acc, s_cf[t], xf(i + s_off[t]));
                epi(i, R(dot2_result(acc)));
            }
        }
    }
}

template <class A, class XF, class EPI>
__device__ __forceinline__ void spmv_dia(const MatView& M, XF xf, EPI epi) {
    __shared__ int s_off[kDiaMax];
    __shared__ double s_c[kDiaMax];
    __shared__ float s_cf[kDiaMax];
    for (int t = threadIdx.x; t < kDiaMax; t += blockDim.x) {
        s_off[t] = t < M.dk ? M.doff[t] : 0;
        s_c[t] = t < M.dk ? M.dc[t] : 0.0;
        s_cf[t] = (float)s_c[t];  // exact: the form requires FP32-exact values
    }
    __syncthreads();
    if (M.dk <= 8) spmv_dia_rows<A, 8>(M, s_off, s_c, s_cf, xf, epi);
    else spmv_dia_rows<A, kDiaMax>(M, s_off, s_c, s_cf, xf, epi);
}

// ---------------------------------------------------------------------------
// Diagonal form in double-float, two rows per thread, over a margined vector.
//
// x (double-float pairs, or FP32 values for the mixed-precision basis) must
// be readable at every index in [-g, n + g) for g > max |offset| + 1; the
// solvers carve such margins around the vectors their levels gather from.
// A thread takes rows i and i + 1 (i even), so a warp covers 64 consecutive
// rows and each offset's two gathers share one address; no index is
// clamped.  A term whose mask bit is clear is replaced by zero before it
// enters the sum, so whatever the margins (or a neighbouring column) hold
// never reaches a result.  epi(i, y0, x0, y1, x1, has1) receives
// y = (A x) and x at rows i and i + 1; has1 is false when i + 1 = n, and then
// y1 and x1 are zero (callers may fold them into sums unconditionally).
//
// Laplacian class (dlap: every off-centre coefficient is dco): the masked
// neighbours are first summed as double-float values (TwoSum of the high
// parts, the low parts and the errors gathered in a second float: 8 FP32
// operations a term), then y = c_centre x_i + dco * sum by one Dot2 step.
// The general case takes each term as a Dot2 step (dot2_add).
template <class TX>
struct DiaVec;

template <>
struct DiaVec<float2> {  // double-float elements
    __device__ static __forceinline__ df64 ld(const float2* p) {
        const float2 v = __ldg(p);
        return df_make(v.x, v.y);
    }
    __device__ static __forceinline__ void ld_pair(const float2* p, df64& a, df64& b) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));  // p at an even index: 16-byte aligned
        a = df_make(v.x, v.y);
        b = df_make(v.z, v.w);
    }
};

template <>
struct DiaVec<float> {  // FP32 elements (exact as double-float)
    __device__ static __forceinline__ df64 ld(const float* p) { return df_make(__ldg(p), 0.f); }
    __device__ static __forceinline__ void ld_pair(const float* p, df64& a, df64& b) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));  // p at an even index: 8-byte aligned
        a = df_make(v.x, 0.f);
        b = df_make(v.y, 0.f);
    }
};

__device__ __forceinline__ void dia_pair_out(df64 c0, df64 c1, int i, int n, const Dot2Acc& a0, const Dot2Acc& a1,
                                             df64& y0, df64& x0, df64& y1, df64& x1, bool& has1) {
    has1 = i + 1 < n;
    x0 = c0;
    y0 = dot2_result(a0);
    x1 = has1 ? c1 : df_make(0.f, 0.f);
    y1 = has1 ? dot2_result(a1) : df_make(0.f, 0.f);
}

template <int K, class TX, class EPI>
__device__ __forceinline__ void spmv_dia_lap(const MatView& M, const TX* __restrict__ x, EPI epi) {
    constexpr int C = K / 2;  // symmetric pattern: offset 0 sits in the middle
    const float cc = (float)M.dc[C], co = M.dco;
    const int n = M.n;
    const int stride = 2 * gridDim.x * blockDim.x;
    // offsets other than the centre and its two neighbours in the sorted order
    // (the +/-1 of a grid): in a warp whose rows all hold them, their terms are
    // summed without the mask select (rows at the grid's far faces are rare;
    // the +/-1 terms stay masked)
    constexpr uint32_t kFar = ((K >= 32 ? 0xffffffffu : ((1u << K) - 1u))) & ~(7u << (C - 1));
    for (int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x); i < n; i += stride) {
        const uint2 mm = __ldg(reinterpret_cast<const uint2*>(M.dmask + i));
        float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f;
        auto sums = [&](auto far_all, auto even) {
#pragma unroll
            for (int t = 0; t < K; t++) {
                if (t == C) continue;
                const TX* a = x + (i + M.doff[t]);
                const bool far = (kFar >> t) & 1u;
                df64 v0, v1;
                if (decltype(even)::value && far) {
                    DiaVec<TX>::ld_pair(a, v0, v1);  // i and the offset even: one aligned pair load
                } else {
                    v0 = DiaVec<TX>::ld(a);
                    v1 = DiaVec<TX>::ld(a + 1);
                }
                const bool all = decltype(far_all)::value && far;
                const bool b0 = all || ((mm.x >> t) & 1u), b1 = all || ((mm.y >> t) & 1u);
                constexpr bool kLo = !std::is_same<TX, float>::value;  // FP32 elements have no low part
                const float h0 = b0 ? v0.hi : 0.f, l0 = kLo && b0 ? v0.lo : 0.f;
                const float h1 = b1 ? v1.hi : 0.f, l1 = kLo && b1 ? v1.lo : 0.f;
                if (t == 0) {  // the first term starts the sums
                    s0 = h0;
                    e0 = l0;
                    s1 = h1;
                    e1 = l1;
                } else {
                    float u, w;
                    two_sum(s0, h0, u, w);
                    s0 = u;
                    e0 = __fadd_rn(e0, kLo ? __fadd_rn(w, l0) : w);
                    two_sum(s1, h1, u, w);
                    s1 = u;
                    e1 = __fadd_rn(e1, kLo ? __fadd_rn(w, l1) : w);
                }
            }
        };
        if (__all_sync(__activemask(), ((mm.x & mm.y) & kFar) == kFar)) {
            if (M.deven) sums(std::true_type{}, std::true_type{});
            else sums(std::true_type{}, std::false_type{});
        } else {
            sums(std::false_type{}, std::false_type{});
        }
        df64 c0, c1;
        DiaVec<TX>::ld_pair(x + i, c0, c1);
        // co * (s + e): its high part exactly as p + fma residue, e scaled into the error float
        float p = __fmul_rn(co, s0);
        Dot2Acc a0{p, __fmaf_rn(co, e0, __fmaf_rn(co, s0, -p))};
        p = __fmul_rn(co, s1);
        Dot2Acc a1{p, __fmaf_rn(co, e1, __fmaf_rn(co, s1, -p))};
        dot2_add(a0, cc, c0);
        dot2_add(a1, cc, c1);
        df64 y0, x0, y1, x1;
        bool has1;
        dia_pair_out(c0, c1, i, n, a0, a1, y0, x0, y1, x1, has1);
        epi(i, y0, x0, y1, x1, has1);
    }
}

template <class TX, class EPI>
__device__ __forceinline__ void spmv_dia_gen(const MatView& M, const TX* __restrict__ x, const int* s_off,
                                             const float* s_cf, EPI epi) {
    const int n = M.n, K = M.dk;
    const int stride = 2 * gridDim.x * blockDim.x;
    const df64 zero = df_make(0.f, 0.f);
    for (int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x); i < n; i += stride) {
        const uint2 mm = __ldg(reinterpret_cast<const uint2*>(M.dmask + i));
        Dot2Acc a0{0.f, 0.f}, a1{0.f, 0.f};
        for (int t = 0; t < K; t++) {
            const TX* a = x + (i + s_off[t]);
            const df64 v0 = DiaVec<TX>::ld(a), v1 = DiaVec<TX>::ld(a + 1);
            const bool b0 = (mm.x >> t) & 1u, b1 = (mm.y >> t) & 1u;
            dot2_add(a0, s_cf[t], b0 ? v0 : zero);
            dot2_add(a1, s_cf[t], b1 ? v1 : zero);
        }
        df64 c0, c1;
        DiaVec<TX>::ld_pair(x + i, c0, c1);
        df64 y0, x0, y1, x1;
        bool has1;
        dia_pair_out(c0, c1, i, n, a0, a1, y0, x0, y1, x1, has1);
        epi(i, y0, x0, y1, x1, has1);
    }
}

// Diagonal-form kernels are built per mode DM (dia_mode() on the host):
// 7 / 27 the Laplacian class with that many offsets, 2 any other diagonal
// form over margined vectors, 1 no margins (clamped, one row per thread,
// each row passed as the first of a pair without a second).  Every thread
// must call it.
template <int DM, class TX, class EPI>
__device__ __forceinline__ void spmv_dia_df(const MatView& M, const TX* __restrict__ x, EPI epi) {
    if constexpr (DM == 7 || DM == 27) {
        spmv_dia_lap<DM>(M, x, epi);
    } else if constexpr (DM == 2) {
        __shared__ int s_off[kDiaMax];
        __shared__ float s_cf[kDiaMax];
        for (int t = threadIdx.x; t < kDiaMax; t += blockDim.x) {
            s_off[t] = t < M.dk ? M.doff[t] : 0;
            s_cf[t] = t < M.dk ? (float)M.dc[t] : 0.f;
        }
        __syncthreads();
        spmv_dia_gen(M, x, s_off, s_cf, epi);
    } else {
        const df64 zero = df_make(0.f, 0.f);
        spmv_dia<ArithDF64>(
            M, [&](int c) { return DiaVec<TX>::ld(x + c); },
            [&](int row, df64 y) { epi(row, y, DiaVec<TX>::ld(x + row), zero, zero, false); });
    }
}

// Minimum resident CTAs per SM the diagonal-form kernels are built for: 6
// (40 registers a thread), except the FP64 forms: the 7-point one gathers two
// rows at a time (4 CTAs, 64 registers), the 27-point one's fixed-point sum
// holds 26 neighbour terms at once (2 CTAs, 128 registers).
template <class A, int DM>
__host__ __device__ constexpr int dia_min_blocks() {
    return (A::kind == 0 && DM == 27) ? 2 : (A::kind == 0 && DM == 7) ? 4 : (DM >= 2 ? 6 : 1);
}

// ---------------------------------------------------------------------------
// Diagonal form in FP64, Laplacian class, over a margined vector.
//
// On a GB300 the FP64 units retire about 2 operations per clock per SM, 1/60
// of the FP32 and 1/40 of the integer rate, so an FP64 stencil row is bound by
// its FP64 operations, not its bytes.  This form spends the fewest: the
// off-centre neighbours (a term whose mask bit is clear replaced by zero with
// an integer select) are summed on the integer units in fixed point
// (fixsum.cuh: one rounding to FP64, error inside that of K - 2 FP64
// additions), or, for the rare row that path declines (NaN or infinity,
// every term below 2^-966, overflow), by K - 2 FP64 additions as a pairwise
// tree; the caller combines the sum S with the centre value in one FMA, e.g.
// D^-1 A x = x + (c_off / d) S for the Jacobi-scaled level.  x must be
// readable at every index in [-g, n + g) for g >= max |offset| (the solvers
// carve such margins).  epi(i, S, x_i) runs once per row, rows grid-stride.
// Sum of the off-centre terms (mask bit t set) of a Laplacian-class row with K
// offsets, offset 0 at index K/2; ld(t) loads the term of offset t as a double.
// The masked neighbours of a Laplacian-class row with K offsets (offset 0 at
// index K/2) as FP64 bit patterns, a term whose mask bit is clear as 0;
// ld(t) loads the term of offset t.
template <int K, class LD>
__device__ __forceinline__ void lap_gather(uint32_t m, LD ld, uint64_t (&w)[K - 1]) {
    constexpr int C = K / 2;
#pragma unroll
    for (int t = 0; t < K; t++) {
        if (t == C) continue;
        const double v = ld(t);
        w[t < C ? t : t - 1] = ((m >> t) & 1u) ? (uint64_t)__double_as_longlong(v) : 0ull;
    }
}

// Their sum: fixed point, or FP64 additions for a row fixsum declines.
template <int K>
__device__ __forceinline__ double lap_sum(const uint64_t (&w)[K - 1]) {
    uint64_t sb;
    if (fixsum<K - 1>(w, &sb)) return __longlong_as_double((long long)sb);
    double d[K - 1];  // the rare row the fixed-point path declines: a pairwise tree of FP64 additions
#pragma unroll
    for (int q = 0; q < K - 1; q++) d[q] = __longlong_as_double((long long)w[q]);
#pragma unroll
    for (int h = 1; h < K - 1; h *= 2) {
#pragma unroll
        for (int q = 0; q + h < K - 1; q += 2 * h) d[q] += d[q + h];
    }
    return d[0];
}

// Sum of the off-centre terms (mask bit t set) of a Laplacian-class row with K
// offsets, offset 0 at index K/2; ld(t) loads the term of offset t as a double.
template <int K, class LD>
__device__ __forceinline__ double lap_neighbour_sum(uint32_t m, LD ld) {
    uint64_t w[K - 1];
    lap_gather<K>(m, ld, w);
    return lap_sum<K>(w);
}

// For the 7-point pattern rows go two at a time per thread (i and i + the
// grid's threads), both rows' loads issued before either row's arithmetic;
// larger patterns take one row at a time.
template <int K, class EPI>
__device__ __forceinline__ void spmv_dia_lap_f64(const MatView& M, const double* __restrict__ x, EPI epi) {
    const int n = M.n;
    const int stride = gridDim.x * blockDim.x;
    if constexpr (K > 7) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const uint32_t m = __ldg(M.dmask + i);
            const double S = lap_neighbour_sum<K>(m, [&](int t) { return __ldg(x + (i + M.doff[t])); });
            epi(i, S, __ldg(x + i));
        }
        return;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
        const int i2 = i + stride;
        const bool two = i2 < n;
        const int j2 = two ? i2 : i;  // a row that exists, for the second gather
        const uint32_t m1 = __ldg(M.dmask + i), m2 = two ? __ldg(M.dmask + j2) : 0u;
        uint64_t w1[K - 1], w2[K - 1];
        lap_gather<K>(m1, [&](int t) { return __ldg(x + (i + M.doff[t])); }, w1);
        lap_gather<K>(m2, [&](int t) { return __ldg(x + (j2 + M.doff[t])); }, w2);
        const double x1 = __ldg(x + i), x2 = __ldg(x + j2);
        const double S1 = lap_sum<K>(w1);
        const double S2 = lap_sum<K>(w2);
        epi(i, S1, x1);
        if (two) epi(i2, S2, x2);
    }
}

// ---------------------------------------------------------------------------
// TMA-pipelined row tiles.
//
// Each CTA walks its tiles (blockIdx.x, +gridDim.x, ...) through NS shared
// memory stages.  Thread 0 fills a stage with three (four for double-float
// values) 1-D bulk copies, cp.async.bulk global -> shared, completing on the
// stage's mbarrier: the tile's row pointers, and the column indices and
// values of its contiguous entry range, widened to 16-byte boundaries (the
// matrix storage carries 16 entries of slack after every array, so the
// widened range never leaves it).  While the CTA computes tile k the copies
// of tiles k+1 .. k+NS-1 are in flight.  Every wait is bounded by
// %globaltimer; on expiry the kernel records SSCG_TIMEOUT, waits (bounded)
// for its own outstanding copies and returns.

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bounded waits give up after 2 s
constexpr int kStages = 2;                        // pipeline depth of the SpMV kernels

// Dynamic shared memory rounded up to a 128-byte boundary (callers size the
// allocation with 128 bytes of slack).
__device__ __forceinline__ char* align128(char* p) {
    return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

// Wait for the phase of `bar` with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (unsigned it = 1; it < (1u << 30); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && globaltimer() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

// Bytes per element of the value arrays a stage holds (second array: the
// low part of double-float values).
template <int VM>
__host__ __device__ constexpr int val0_bytes() { return VM == VAL_F64 ? 8 : 4; }
template <int VM>
__host__ __device__ constexpr int val1_bytes() { return VM == VAL_DF ? 4 : 0; }

constexpr int kPipeRp = kTileRows + 4;  // row-pointer slots per stage (multiple of 4)

template <int VM>
__host__ __device__ constexpr size_t pipe_stage_bytes(int cap) {
    return (size_t)kPipeRp * 4 + (size_t)cap * (4 + val0_bytes<VM>() + val1_bytes<VM>());
}

template <int VM, int NS>
__host__ __device__ constexpr size_t pipe_bytes(int cap) {
    return 16 * ((NS * 8 + 15) / 16) + NS * pipe_stage_bytes<VM>(cap);
}

template <class A, int VM>
__device__ __forceinline__ typename Val<A, VM>::T stage_val(const char* v0, const char* v1, int k);

template <>
__device__ __forceinline__ double stage_val<ArithF64, VAL_F64>(const char* v0, const char*, int k) {
    return reinterpret_cast<const double*>(v0)[k];
}
template <>
__device__ __forceinline__ float stage_val<ArithDF64, VAL_F32>(const char* v0, const char*, int k) {
    return reinterpret_cast<const float*>(v0)[k];
}
template <>
__device__ __forceinline__ float stage_val<ArithF32, VAL_F32>(const char* v0, const char*, int k) {
    return reinterpret_cast<const float*>(v0)[k];
}
template <>
__device__ __forceinline__ float2 stage_val<ArithDF64, VAL_DF>(const char* v0, const char* v1, int k) {
    return make_float2(reinterpret_cast<const float*>(v0)[k], reinterpret_cast<const float*>(v1)[k]);
}

// Thread 0: bulk-copy tile t's row pointers, column indices and values into
// the stage at `st`, completing on `bar`.
template <int VM>
__device__ __forceinline__ void issue_tile(const MatView& M, char* st, uint64_t* bar, int t) {
    const int cap = M.cap;
    const int r0 = t * kTileRows, nrows = min(kTileRows, M.n - r0);
    const int lo = __ldg(M.rowptr + r0), hi = __ldg(M.rowptr + r0 + nrows);
    const int base = lo & ~3, end = min((hi + 3) & ~3, base + cap), cnt = end - base;
    const unsigned rpb = (unsigned)(((nrows + 1 + 3) & ~3) * 4);
    const unsigned tx = rpb + (unsigned)cnt * (4 + val0_bytes<VM>() + val1_bytes<VM>());
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, tx);
    bulk_g2s(st, M.rowptr + r0, rpb, bar);
    if (cnt > 0) {
        char* cdst = st + kPipeRp * 4;
        char* v0 = cdst + (size_t)cap * 4;
        bulk_g2s(cdst, M.col + base, (unsigned)cnt * 4, bar);
        if (VM == VAL_F64) bulk_g2s(v0, M.val + base, (unsigned)cnt * 8, bar);
        else bulk_g2s(v0, M.vhi + base, (unsigned)cnt * 4, bar);
        if (VM == VAL_DF) bulk_g2s(v0 + (size_t)cap * 4, M.vlo + base, (unsigned)cnt * 4, bar);
    }
}

// Every thread: row r0 + threadIdx.x of tile t from the staged data (entries
// past the stage's capacity from global memory); epi(row, y).
template <class A, int VM, class XF, class EPI>
__device__ __forceinline__ void compute_tile(const MatView& M, const char* st, int t, XF xf, EPI epi) {
    using V = Val<A, VM>;
    const int cap = M.cap;
    const int* s_rp = reinterpret_cast<const int*>(st);
    const int32_t* s_col = reinterpret_cast<const int32_t*>(st + kPipeRp * 4);
    const char* v0 = st + kPipeRp * 4 + (size_t)cap * 4;
    const char* v1 = v0 + (size_t)cap * val0_bytes<VM>();
    const int r0 = t * kTileRows, nrows = min(kTileRows, M.n - r0);
    const int base = s_rp[0] & ~3;
    const int staged = min((s_rp[nrows] + 3) & ~3, base + cap) - base;
    if ((int)threadIdx.x < nrows) {
        const int ks = s_rp[threadIdx.x] - base, ke = s_rp[threadIdx.x + 1] - base;
        const int km = min(ke, staged);
        typename A::R y = A::zero();
        for (int q = ks; q < km; q++) y = V::mac(y, stage_val<A, VM>(v0, v1, q), xf(s_col[q]));
        for (int q = max(ks, staged); q < ke; q++) y = V::mac(y, V::load(M, base + q), xf(__ldg(M.col + base + q)));
        epi(r0 + (int)threadIdx.x, y);
    }
}

// Runs epi(row, y) with y = (A x)[row] for every row of this CTA's tiles.
// M.cap (a multiple of 4) is the entries a stage holds.  Every thread of the
// CTA must call it; `smem` holds pipe_bytes<VM, NS>(M.cap).  Returns false
// after a timeout (recorded in ctrl).
template <class A, int VM, int NS, class XF, class EPI>
__device__ __forceinline__ bool spmv_pipe(const MatView& M, char* smem, XF xf, EPI epi, Ctrl* ctrl) {
    const int cap = M.cap;
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    const int G = gridDim.x;
    const int my = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + G - 1) / G : 0;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    char* stage0 = smem + 16 * ((NS * 8 + 15) / 16);
    const size_t sb = pipe_stage_bytes<VM>(cap);
    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; q++) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int k) {  // thread 0: tile k of this CTA into stage k % NS
        issue_tile<VM>(M, stage0 + (size_t)(k % NS) * sb, &bar[k % NS], (int)blockIdx.x + k * G);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < NS - 1 && k < my; k++) issue(k);
    for (int k = 0; k < my; k++) {
        if (threadIdx.x == 0 && k + NS - 1 < my) issue(k + NS - 1);
        const bool ok = __syncthreads_and(mbar_wait(&bar[k % NS], (unsigned)(k / NS) & 1u));
        if (!ok) {
            if (threadIdx.x == 0) {
                ctrl->status = 3;  // SSCG_TIMEOUT
                __threadfence();
                atomicExch(&ctrl->done, 1);
                for (int q = k + 1; q < my && q < k + NS; q++) mbar_wait(&bar[q % NS], (unsigned)(q / NS) & 1u);
            }
            __syncthreads();
            return false;
        }
        compute_tile<A, VM>(M, stage0 + (size_t)(k % NS) * sb, (int)blockIdx.x + k * G, xf, epi);
        __syncthreads();  // stage k % NS may be refilled
    }
    return true;
}

}  // namespace sscg
