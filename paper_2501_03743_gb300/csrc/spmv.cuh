// CSR row-tile SpMV shared by every kernel that multiplies by A.
//
// A CTA takes a tile of kTileRows consecutive rows.  It loads the tile's
// row pointers, then copies the tile's contiguous column-index and value
// ranges into shared memory with coalesced loads, and each thread forms the
// dot product of one row from shared memory, gathering x[col] through the
// read-only cache.  Tiles whose entries exceed the staging capacity take the
// remainder straight from global memory.
#pragma once

#include "common.cuh"

namespace sscg {

// How the matrix values are stored and multiplied.
enum ValMode { VAL_F64 = 0, VAL_F32 = 1, VAL_DF = 2 };

struct MatView {
    int n;
    int cap;  // staging capacity (entries) of the dynamic shared memory
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ col;
    const double* __restrict__ val;
    const float* __restrict__ vhi;
    const float* __restrict__ vlo;
};

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

}  // namespace sscg
