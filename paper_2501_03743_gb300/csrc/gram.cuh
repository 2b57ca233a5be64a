// Basis and Gram kernels of the direct-Gram s-step path, shared by the
// DF64/F64 driver (sstep_gram.cu) and the mixed-precision driver (mixed.cu).
#pragma once

#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "small.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

// Basis recurrence coefficients with w = B^-1 A u_j: monomial u_{j+1} = w;
// Chebyshev u_2 = (w - c u_1)/delta, u_{j+1} = 2 (w - c u_j)/delta - u_{j-1};
// Newton u_{j+1} = (w - theta_j u_j) / sigma.
struct Basis {
    int cheb;
    int newton;
    double c, delta;
    double theta[kMaxS];  // Newton shifts theta_0 .. theta_{s-2}
    double isig;          // 1 / sigma
};

// The basis of a solve over the interval [lo, hi] of B^-1 A.  Newton shifts
// (Section IV names the Newton basis; the shift choice is this library's):
// the s - 1 Chebyshev points of [lo, hi] (zeros of T_{s-1}) in Leja order,
// each next point the one whose distances to the points already taken have
// the largest product (the first: the largest in modulus; scores within
// 1e-12 relative of each other go to the lower index), with the scale
// sigma = (hi - lo)/4, the capacity of the interval, which keeps the basis
// vectors' norms of the order of the first one's.
inline Basis make_basis(int kind, int s, double lo, double hi) {
    Basis b{};
    b.cheb = kind == SSCG_BASIS_CHEBYSHEV;
    b.newton = kind == SSCG_BASIS_NEWTON;
    b.c = 0.5 * (hi + lo);
    b.delta = 0.5 * (hi - lo);
    b.isig = 1.0;
    if (b.newton && s > 1 && b.delta > 0.0) {
        const int m = s - 1;
        double pts[kMaxS];
        bool taken[kMaxS] = {};
        for (int k = 0; k < m; k++) pts[k] = b.c + b.delta * std::cos(M_PI * (2 * k + 1) / (2.0 * m));
        for (int q = 0; q < m; q++) {
            int pick = -1;
            double best = -1.0;
            for (int k = 0; k < m; k++) {
                if (taken[k]) continue;
                double score = std::fabs(pts[k]);
                if (q > 0) {
                    score = 1.0;
                    for (int i = 0; i < q; i++) score *= std::fabs(pts[k] - b.theta[i]);
                }
                if (pick < 0 || score > best * (1.0 + 1e-12)) best = score, pick = k;  // near-ties: lower k
            }
            taken[pick] = true;
            b.theta[q] = pts[pick];
        }
        b.isig = 4.0 / (hi - lo);
    }
    return b;
}

template <class A>
__device__ __forceinline__ typename A::R basis_next(const Basis& B, int j, typename A::R w,
                                                    const typename A::S* uj, const typename A::S* ujm1, int row) {
    if (B.newton)
        return A::mul(A::sub(w, A::mul(A::from_d(B.theta[j]), A::ld(uj + row))), A::from_d(B.isig));
    if (!B.cheb) return w;
    typename A::R t = A::sub(w, A::mul(A::from_d(B.c), A::ld(uj + row)));
    if (j == 0) return A::mul(t, A::from_d(1.0 / B.delta));
    return A::sub(A::mul(t, A::from_d(2.0 / B.delta)), A::ld(ujm1 + row));
}

// AU_j = A u_j; with a diagonal preconditioner also u_{j+1}.  The matrix in
// CSR tiles or, with DM != 0 (double-float only), its diagonal form (mode DM
// of spmv_dia_df); there B^-1 is the constant dinv_c (Jacobi) or the identity
// (dinv_c = 0), and the vectors gathered carry margins.
template <class A, int VM, int DM = 0>
__global__ void __launch_bounds__(kThreads, DM >= 2 ? 6 : 1)
    k_level_gen(MatView M, const typename A::S* __restrict__ dinv, double dinv_c,
                const typename A::S* __restrict__ u_in, const typename A::S* __restrict__ u_prev,
                typename A::S* __restrict__ au_out, typename A::S* __restrict__ u_next, int j, Basis B,
                int diag_prec, const Ctrl* ctrl) {
    using R = typename A::R;
    if (ctrl_done(ctrl)) return;
    if constexpr (DM != 0 && A::kind == 1) {
        const df64 dcv = dinv_c != 0.0 ? df_from_double(dinv_c) : df_make(1.f, 0.f);
        const df64 cb = df_from_double(B.c);
        const df64 sc = df_from_double(B.cheb ? (j == 0 ? 1.0 : 2.0) / B.delta : 1.0);
        const bool nxt = u_next && diag_prec;
        spmv_dia_df<DM>(M, u_in, [&](int i, df64 y0, df64 x0, df64 y1, df64 x1, bool has1) {
            if (has1) st_pair(au_out + i, y0, y1);
            else A::st(au_out + i, y0);
            if (!nxt) return;
            df64 w0 = df_mul(dcv, y0), w1 = df_mul(dcv, y1);
            if (B.newton) {  // Newton recurrence on w = B^-1 A u_j
                const df64 th = df_from_double(B.theta[j]), is = df_from_double(B.isig);
                w0 = df_mul(df_add(w0, df_neg(df_mul(th, x0))), is);
                w1 = df_mul(df_add(w1, df_neg(df_mul(th, x1))), is);
            } else if (B.cheb) {  // Chebyshev recurrence on w = B^-1 A u_j
                w0 = df_mul(df_add(w0, df_neg(df_mul(cb, x0))), sc);
                w1 = df_mul(df_add(w1, df_neg(df_mul(cb, x1))), sc);
                if (j > 0) {
                    df64 p0, p1;
                    DiaVec<float2>::ld_pair(u_prev + i, p0, p1);
                    w0 = df_add(w0, df_neg(p0));
                    w1 = df_add(w1, df_neg(p1));
                }
            }
            if (has1) st_pair(u_next + i, w0, w1);
            else A::st(u_next + i, w0);
        });
    } else {
        extern __shared__ __align__(16) char smem_raw[];
        char* smem = align128(smem_raw);
        spmv_pipe<A, VM, kStages>(
            M, smem, [&](int c) { return A::ldg(u_in + c); },
            [&](int row, R y) {
                A::st(au_out + row, y);
                if (u_next && diag_prec) {
                    R w = dinv ? A::mul(A::ld(dinv + row), y) : y;
                    A::st(u_next + row, basis_next<A>(B, j, w, u_in, u_prev, row));
                }
            },
            const_cast<Ctrl*>(ctrl));
    }
}

// u_{j+1} from w = B^-1 A u_j (general preconditioner).
template <class A>
__global__ void __launch_bounds__(kThreads) k_combine(int n, const typename A::S* __restrict__ w,
                                                      const typename A::S* __restrict__ u_in,
                                                      const typename A::S* __restrict__ u_prev,
                                                      typename A::S* __restrict__ u_next, int j, Basis B,
                                                      const Ctrl* ctrl) {
    if (ctrl_done(ctrl)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        A::st(u_next + i, basis_next<A>(B, j, A::ld(w + i), u_in, u_prev, i));
}

// Gram entries: e < ng: G(i, j), i >= j (u_i . AU_j); then m(i) (u_i . r);
// then C(l, j) ((A p_l^old) . u_j) when a previous block exists.
// then, with a true (replaced) residual, q(l) = p_l^old . r.
// with_q = 2 (cp): C(l, j) is formed as p_l^old . (A u_j), equal for a
// symmetric A, so the previous block's A P is not needed.
struct GramShape {
    int s, ng, nm, nc, nq, E, ncols, cp;
};

__host__ __device__ inline GramShape gram_shape(int s, int has_old, int with_q = 0) {
    GramShape g;
    g.s = s;
    g.ng = s * (s + 1) / 2;
    g.nm = s;
    g.nc = has_old ? s * s : 0;
    g.nq = (has_old && with_q) ? s : 0;
    g.cp = (has_old && with_q == 2) ? 1 : 0;
    g.E = g.ng + g.nm + g.nc + g.nq;
    g.ncols = g.cp ? 3 * s + 1 : 2 * s + 1 + (has_old ? s : 0) + g.nq;
    return g;
}

// Columns staged per tile: U_0..U_{s-1}, AU_0..AU_{s-1}, r,
// AP_old_0..AP_old_{s-1}, P_old_0..P_old_{s-1} (cp: U, AU, r, P_old).
__device__ __forceinline__ void gram_entry(const GramShape& g, int e, int& a, int& b) {
    const int s = g.s;
    if (e < g.ng) {  // lower-triangle index -> (i, j), i >= j
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= e) i++;
        int j = e - i * (i + 1) / 2;
        a = i;
        b = s + j;
    } else if (e < g.ng + g.nm) {
        a = e - g.ng;
        b = 2 * s;
    } else if (e < g.ng + g.nm + g.nc) {
        int q = e - g.ng - g.nm;
        int l = q % s, j = q / s;
        a = 2 * s + 1 + l;
        b = g.cp ? s + j : j;
    } else {
        int l = e - g.ng - g.nm - g.nc;
        a = (g.cp ? 2 * s + 1 : 3 * s + 1) + l;
        b = 2 * s;
    }
}

constexpr int kGramTile = 128;  // rows staged per tile

// Asynchronous global -> shared element copies (cp.async), zero-filled past
// src_bytes; completion tracked per thread by commit groups.
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// TB: element type of the basis columns U (the new block's first s
// columns, or `ublk` when given); AU (`au`, s columns), r and the old block
// use A::S.  The mixed-precision mode passes FP32 U with FP64 AU, r and
// P_old (A = ArithF64: the FP32 elements are widened in shared memory).
template <class A, int SB, class TB = typename A::S>
__global__ void __launch_bounds__(kThreads) k_gram(int n, int ldn, int s, const typename A::S* __restrict__ blk_new,
                                                   const TB* __restrict__ ublk, const typename A::S* __restrict__ au,
                                                   const typename A::S* __restrict__ r,
                                                   const typename A::S* __restrict__ blk_old, int has_old,
                                                   int with_q, double* __restrict__ part, int step, Ctrl* ctrl) {
    using R = typename A::R;
    using S = typename A::S;
    if (ctrl_done(ctrl)) return;
    extern __shared__ __align__(16) char smem[];
    S* tile = reinterpret_cast<S*>(smem);  // [ncols][kGramTile + 1]
    constexpr int LD = kGramTile + 1;
    const GramShape g = gram_shape(s, has_old, with_q);
    // thread -> (entry, row group); entries beyond the thread count loop
    const int groups = g.E >= kThreads ? 1 : kThreads / g.E;
    const int active = g.E >= kThreads ? kThreads : g.E * groups;
    constexpr int kMaxEPT = (SB * (SB + 1) / 2 + 2 * SB + SB * SB + kThreads - 1) / kThreads;
    int ea[kMaxEPT], eb[kMaxEPT];
    R acc[kMaxEPT];
    const int grp = threadIdx.x / (g.E >= kThreads ? kThreads : g.E);
    const int e0 = threadIdx.x % (g.E >= kThreads ? kThreads : g.E);
#pragma unroll
    for (int q = 0; q < kMaxEPT; q++) {
        acc[q] = A::zero();
        int e = e0 + q * kThreads;
        if (e < g.E) gram_entry(g, e, ea[q], eb[q]);
        else ea[q] = eb[q] = 0;
    }
    const size_t ld = (size_t)ldn;
    const int ntiles = (n + kGramTile - 1) / kGramTile;
    // Two tile buffers: the next tile's columns are copied global -> shared by
    // cp.async (8 bytes an element; 4 for an FP32 basis element, whose low
    // float stays zero) while the current one is summed.  Rows past n are
    // zero-filled by the copies themselves.
    const int tstride = g.ncols * LD;
    if (ublk) {
        for (int idx = threadIdx.x; idx < 2 * s * LD; idx += blockDim.x) {
            const int bsel = idx / (s * LD), rem = idx % (s * LD);
            reinterpret_cast<float*>(tile + bsel * tstride + rem)[1] = 0.f;
        }
    }
    // column bases, once per CTA; a thread then copies one fixed row of a tile
    // (i = threadIdx.x mod 128) for every second column (blockDim.x = 256)
    __shared__ const void* s_src[4 * kMaxS + 2];
    for (int c = threadIdx.x; c < g.ncols; c += blockDim.x) {
        const void* p;
        if (c < s) p = ublk ? static_cast<const void*>(ublk + c * ld) : static_cast<const void*>(blk_new + c * ld);
        else if (c < 2 * s) p = au + (c - s) * ld;
        else if (c == 2 * s) p = r;
        else if (g.cp) p = blk_old + (c - 2 * s - 1) * ld;  // P_old
        else if (c <= 3 * s) p = blk_old + (s + (c - 2 * s - 1)) * ld;
        else p = blk_old + (c - 3 * s - 1) * ld;
        s_src[c] = p;
    }
    __syncthreads();
    auto stage = [&](int t, int b) {
        const int i = threadIdx.x % kGramTile, row = t * kGramTile + i;
        const int ok = row < n;
        const size_t rr = ok ? (size_t)row : 0;
        S* dst = tile + b * tstride + i;
        for (int c = threadIdx.x / kGramTile; c < g.ncols; c += blockDim.x / kGramTile) {
            if (ublk && c < s) cp_async4(dst + c * LD, static_cast<const TB*>(s_src[c]) + rr, ok ? 4 : 0);
            else cp_async8(dst + c * LD, static_cast<const S*>(s_src[c]) + rr, ok ? 8 : 0);
        }
    };
    int buf = 0;
    if (blockIdx.x < ntiles) stage(blockIdx.x, 0);
    cp_async_commit();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (t + (int)gridDim.x < ntiles) stage(t + gridDim.x, buf ^ 1);
        cp_async_commit();
        cp_async_wait_prior();  // every group but the newest: tile t is in
        __syncthreads();
        if constexpr (A::kind == 0 && std::is_same<TB, float>::value) {
            // FP64 sums of an FP32 basis: each thread widens the U elements it
            // staged (the low 4 bytes of their slots) to FP64 in place
            if (ublk) {
                const int i = threadIdx.x % kGramTile;
                for (int c = threadIdx.x / kGramTile; c < s; c += blockDim.x / kGramTile) {
                    S* d = tile + buf * tstride + c * LD + i;
                    *d = (double)reinterpret_cast<const float*>(d)[0];
                }
                __syncthreads();
            }
        }
        const S* tile_t = tile + buf * tstride;
        if (threadIdx.x < active) {
#pragma unroll
            for (int q = 0; q < kMaxEPT; q++) {
                if (e0 + q * kThreads >= g.E) break;
                const S* ta = tile_t + ea[q] * LD;
                const S* tb = tile_t + eb[q] * LD;
                R a = acc[q];
                for (int i = grp; i < kGramTile; i += groups) a = A::fma(A::ld(ta + i), A::ld(tb + i), a);
                acc[q] = a;
            }
        }
        __syncthreads();  // tile t is read: its buffer takes tile t + 2 gridDim.x next
        buf ^= 1;
    }
    cp_async_wait_all();
    // combine the row groups of each entry, then one partial per entry
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem);  // kThreads doubles (tile is free now)
    const int G = gridDim.x;
#pragma unroll
    for (int q = 0; q < kMaxEPT; q++) {
        red[threadIdx.x] = (threadIdx.x < active) ? A::to_d(acc[q]) : 0.0;
        __syncthreads();
        int e = e0 + q * kThreads;
        if (grp == 0 && threadIdx.x < active && e < g.E) {
            double t = 0.0;
            for (int gg = 0; gg < groups; gg++) t += red[e0 + gg * (g.E >= kThreads ? kThreads : g.E)];
            part[(size_t)e * G + blockIdx.x] = t;
        }
        __syncthreads();
    }
    if (!last_cta(&ctrl->ticket[1])) return;
    cta_sum_rows(part, g.E, G, [&](int e, double v) {
        int a, b;
        gram_entry(g, e, a, b);
        if (e < g.ng) {
            int i = a, j = b - s;
            ctrl->G[i + j * s] = v;
            ctrl->G[j + i * s] = v;
        } else if (e < g.ng + g.nm) {
            ctrl->m[a] = v;
        } else if (e < g.ng + g.nm + g.nc) {
            int l = a - 2 * s - 1, j = g.cp ? b - s : b;
            ctrl->C[l + j * s] = v;
        } else {
            ctrl->q[a - (g.cp ? 2 * s + 1 : 3 * s + 1)] = v;
        }
    });
    if (threadIdx.x == 0) ctrl->with_q = g.nq > 0;
    __syncthreads();
    SmallScratch* sc = reinterpret_cast<SmallScratch*>(smem);
    if (threadIdx.x < 32) {
        int st = warp_sw_gram(ctrl, s, step, sc);
        if (threadIdx.x == 0 && st != 0) {
            ctrl->status = st;
            ctrl->done = 1;
        }
    }
}

}  // namespace

}  // namespace sscg
