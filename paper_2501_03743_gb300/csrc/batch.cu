// Batched s-step CG: many independent SPD systems, each with 1..8 right-hand
// sides, solved by one persistent cooperative kernel.
//
// Every system runs Algorithm 3 with the monomial basis, the Jacobi
// preconditioner and the moment recurrence of Algorithm 6, per right-hand
// side, as the single-system path does.  The kernel walks the phases of an
// outer step for all systems at once, separated by grid-wide barriers:
//
//   level j = 0..s-1   matrix-powers level (Algorithm 4) of every active
//                      system: AU_j = A U_j, U_{j+1} = D^-1 AU_j for all its
//                      right-hand sides in one pass over the matrix (SpMM),
//                      moment partials mu_{2j+1}, mu_{2j+2} per item
//   solve              per system (one CTA): reduce the partials, test
//                      convergence, run Algorithm 6 per right-hand side
//                      (one warp each)
//   update             block updates of Algorithm 3 plus z = D^-1 r and the
//                      partials of ||r||^2 and mu_0 for the next step
//
// Work is divided into items of T consecutive rows of one system (T chosen
// per size class, by the autotuner when asked); CTA c takes items c, c+G,
// ...  Vectors hold a system's right-hand sides interleaved (row i, rhs r
// at i*R + r) so one gather of A's column serves all of them.  A system
// whose right-hand sides are all done exports x = x0 + correction in the
// next update phase, forms its true residual in the next level-0 phase and
// is finished (device timestamp recorded) in the next solve phase, so each
// system's result is final as soon as it converges.
//
// Barrier waits are bounded by %globaltimer: on expiry the kernel records
// SSCG_TIMEOUT and every CTA returns.  Data produced inside the kernel is
// read through L2 (ld.global.cg); the matrix through the read-only path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "small.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

constexpr int kMaxR = SSCG_BATCH_MAX_RHS;
constexpr int kMaxSB = SSCG_BATCH_MAX_S;
constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;
constexpr int kTileCand[] = {256, 512, 1024, 2048, 4096};
constexpr int kNumCand = 5;
constexpr int kMinTile = 256;
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;

enum SysState { SYS_ACTIVE = 0, SYS_EXPORT = 1, SYS_FINISHED = 2 };

struct BSys {
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    const float* vhi;
    const float* vlo;
    const void* dinv;  // double (F64) or float2 (double-float)
    void* blk[2];      // 2s columns of n x R each: U | AU, later P | AP
    void* xw;          // correction to x0, n x R
    void* r;           // residual, n x R
    double* lpart;     // (2s-1) R rows of `items` moment partials
    double* upart;     // 3 R rows: ||r||^2, mu_0, ||b||^2 (step 0) / true residual^2
    int n, R, exact, T;
    int items, item0, rhs0, pad;
};

struct GridBar {
    unsigned count;
    unsigned gen;
};

struct GCtl {
    GridBar bar;
    int err;
    int finished;
    unsigned long long t0;
};

struct BCtl {
    int state;
    int step;  // outer steps whose coefficients have been computed
    unsigned long long t_fin;
};

struct BArgs {
    int nsys, nitems, s, maxit, tuning;
    double tol;
    const BSys* sys;
    const int* item_sys;
    const double* const* io;  // B[k] at io[2k], X[k] at io[2k+1]
    GCtl* g;
    BCtl* bctl;
    Ctrl* rc;  // one per right-hand side
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier (all CTAs are co-resident: cooperative launch).  Returns
// false when the kernel must stop (a wait expired here or elsewhere).
__device__ bool grid_sync(GCtl* g) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_gpu(&g->bar.gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&g->bar.count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&g->bar.count, 0u);
            __threadfence();
            st_release_gpu(&g->bar.gen, gen + 1);
        } else {
            const uint64_t t0 = globaltimer();
            while (ld_acquire_gpu(&g->bar.gen) == gen) {
                if (*(volatile int*)&g->err) {
                    ok = 0;
                    break;
                }
                if (globaltimer() - t0 > kBarrierTimeoutNs) {
                    atomicCAS(&g->err, 0, SSCG_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile int*)&g->err) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ double splitmix_u(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1p-52 - 1.0;
}

template <class A>
struct BK {
    using Rv = typename A::R;
    using S = typename A::S;

    static __device__ __forceinline__ S* col(void* base, int c, const BSys& y) {
        return reinterpret_cast<S*>(base) + (size_t)c * y.n * y.R;
    }

    // Load the R interleaved values of row i of an n x R vector (data written
    // in this kernel: through L2).
    static __device__ __forceinline__ void ld_row(const S* v, int i, int R, Rv (&out)[kMaxR]) {
        const S* p = v + (size_t)i * R;
#pragma unroll
        for (int r = 0; r < kMaxR; r++)
            if (r < R) out[r] = A::ldcg(p + r);
    }

    static __device__ __forceinline__ Rv dinv_of(const BSys& y, int i) {
        return A::ldg(reinterpret_cast<const S*>(y.dinv) + i);
    }

    // acc[r] = (A v_r)[i] for the R interleaved vectors v (device, this kernel).
    static __device__ __forceinline__ void spmm_row(const BSys& y, int i, const S* v, Rv (&acc)[kMaxR]) {
        const int R = y.R;
#pragma unroll
        for (int r = 0; r < kMaxR; r++) acc[r] = A::zero();
        const int k0 = __ldg(y.rowptr + i), k1 = __ldg(y.rowptr + i + 1);
        for (int k = k0; k < k1; k++) {
            const int c = __ldg(y.col + k);
            const S* p = v + (size_t)c * R;
            if constexpr (A::kind == 1) {
                if (y.exact) {
                    const float a = __ldg(y.vhi + k);
#pragma unroll
                    for (int r = 0; r < kMaxR; r++)
                        if (r < R) acc[r] = df_fma_f(A::ldcg(p + r), a, acc[r]);
                } else {
                    const df64 a = df_make(__ldg(y.vhi + k), __ldg(y.vlo + k));
#pragma unroll
                    for (int r = 0; r < kMaxR; r++)
                        if (r < R) acc[r] = df_fma(A::ldcg(p + r), a, acc[r]);
                }
            } else {
                const double a = __ldg(y.val + k);
#pragma unroll
                for (int r = 0; r < kMaxR; r++)
                    if (r < R) acc[r] = ::fma(a, A::ldcg(p + r), acc[r]);
            }
        }
    }

    // acc[r] = (A x_r)[i] for FP64 column-major user vectors X (n x R).
    static __device__ __forceinline__ void spmm_row_user(const BSys& y, int i, const double* X, Rv (&acc)[kMaxR]) {
        const int R = y.R;
#pragma unroll
        for (int r = 0; r < kMaxR; r++) acc[r] = A::zero();
        const int k0 = __ldg(y.rowptr + i), k1 = __ldg(y.rowptr + i + 1);
        for (int k = k0; k < k1; k++) {
            const int c = __ldg(y.col + k);
            Rv a;
            if constexpr (A::kind == 1) a = y.exact ? df_make(__ldg(y.vhi + k), 0.f) : df_make(__ldg(y.vhi + k), __ldg(y.vlo + k));
            else a = __ldg(y.val + k);
#pragma unroll
            for (int r = 0; r < kMaxR; r++)
                if (r < R) acc[r] = A::fma(a, A::from_d(__ldcg(X + (size_t)r * y.n + c)), acc[r]);
        }
    }
};

// Sum NV per-thread values over the CTA in a fixed order; thread q < NV
// receives sum q.  sh holds kMaxR*2 x kBWarps doubles.
template <class A>
__device__ __forceinline__ void cta_sum_n(typename A::R* v, int NV, double (*sh)[kBWarps], double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < NV; q++) {
        typename A::R w = warp_sum<A>(v[q]);
        if (lane == 0) sh[q][warp] = A::to_d(w);
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < kBWarps; w++) t += sh[threadIdx.x][w];
        *out = t;
    }
    __syncthreads();
}

template <class A>
__global__ void __launch_bounds__(kBThreads, 2) k_batch(BArgs a) {
    using K = BK<A>;
    using Rv = typename A::R;
    using S = typename A::S;
    __shared__ double red[2 * kMaxR][kBWarps];
    __shared__ double sw_red[(2 * kMaxSB + 2) * kMaxR];
    __shared__ SmallScratchT<kMaxSB> scratch[kBWarps];
    __shared__ double s_alpha[kMaxR][kMaxSB];
    __shared__ double s_beta[kMaxR][kMaxSB * kMaxSB];
    __shared__ int s_act[kMaxR];
    const int s = a.s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.g->t0 = globaltimer();

    // ---------------------------------------------------------- init
    // r = b - A x0, z = D^-1 r = U_0, correction 0; partials ||r||^2, mu_0, ||b||^2
    for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
        const int k = __ldg(a.item_sys + it);
        const BSys& y = a.sys[k];
        const int li = it - y.item0, R = y.R;
        const int r0 = li * y.T, r1 = min(y.n, r0 + y.T);
        const double* B = a.tuning ? nullptr : a.io[2 * k];
        const double* X = a.tuning ? nullptr : a.io[2 * k + 1];
        Rv rr[kMaxR], rz[kMaxR], bb[kMaxR];
#pragma unroll
        for (int r = 0; r < kMaxR; r++) rr[r] = rz[r] = bb[r] = A::zero();
        S* u0 = K::col(y.blk[0], 0, y);
        S* rv = reinterpret_cast<S*>(y.r);
        S* xw = reinterpret_cast<S*>(y.xw);
        for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) {
            Rv ax[kMaxR];
            if (X) K::spmm_row_user(y, i, X, ax);
            else
#pragma unroll
                for (int r = 0; r < kMaxR; r++) ax[r] = A::zero();
            const Rv di = K::dinv_of(y, i);
#pragma unroll
            for (int r = 0; r < kMaxR; r++) {
                if (r >= R) continue;
                const double bv = B ? __ldg(B + (size_t)r * y.n + i) : splitmix_u(0xBA7C5EEDull + k, (size_t)i * R + r);
                const Rv b = A::from_d(bv);
                const Rv res = A::sub(b, ax[r]);
                const Rv z = A::mul(di, res);
                A::st(rv + (size_t)i * R + r, res);
                A::st(u0 + (size_t)i * R + r, z);
                A::st(xw + (size_t)i * R + r, A::zero());
                rr[r] = A::fma(res, res, rr[r]);
                rz[r] = A::fma(res, z, rz[r]);
                bb[r] = A::fma(b, b, bb[r]);
            }
        }
        Rv v[3 * kMaxR];
        for (int r = 0; r < R; r++) {
            v[r] = rr[r];
            v[R + r] = rz[r];
            v[2 * R + r] = bb[r];
        }
        double out = 0.0;
        // 3R <= 24 values: two passes through the 2*kMaxR-row buffer
        cta_sum_n<A>(v, 2 * R, red, &out);
        if (threadIdx.x < 2 * R) y.upart[(size_t)threadIdx.x * y.items + li] = out;
        cta_sum_n<A>(v + 2 * R, R, red, &out);
        if (threadIdx.x < R) y.upart[(size_t)(2 * R + threadIdx.x) * y.items + li] = out;
    }
    if (!grid_sync(a.g)) return;

    for (int outer = 0;; outer++) {
        // ------------------------------------------------------ levels
        for (int j = 0; j < s; j++) {
            for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
                const int k = __ldg(a.item_sys + it);
                const BSys& y = a.sys[k];
                const int state = __ldcg(&a.bctl[k].state);
                if (state == SYS_FINISHED || (state == SYS_EXPORT && (j > 0 || a.tuning))) continue;
                const int li = it - y.item0, R = y.R;
                const int r0 = li * y.T, r1 = min(y.n, r0 + y.T);
                if (state == SYS_EXPORT) {
                    // true residual of the exported x: b - A x
                    const double* B = a.io[2 * k];
                    const double* X = a.io[2 * k + 1];
                    Rv tr[kMaxR];
#pragma unroll
                    for (int r = 0; r < kMaxR; r++) tr[r] = A::zero();
                    for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) {
                        Rv ax[kMaxR];
                        K::spmm_row_user(y, i, X, ax);
#pragma unroll
                        for (int r = 0; r < kMaxR; r++) {
                            if (r >= R) continue;
                            const Rv e = A::sub(A::from_d(__ldg(B + (size_t)r * y.n + i)), ax[r]);
                            tr[r] = A::fma(e, e, tr[r]);
                        }
                    }
                    double out = 0.0;
                    cta_sum_n<A>(tr, R, red, &out);
                    if (threadIdx.x < R) y.upart[(size_t)(2 * R + threadIdx.x) * y.items + li] = out;
                    continue;
                }
                const int step = __ldcg(&a.bctl[k].step);
                void* blk = y.blk[step & 1];
                const S* uj = K::col(blk, j, y);
                S* au = K::col(blk, s + j, y);
                S* un = j < s - 1 ? K::col(blk, j + 1, y) : nullptr;
                const bool want_m2 = 2 * j + 2 <= 2 * s - 1;
                Rv m1[kMaxR], m2[kMaxR];
#pragma unroll
                for (int r = 0; r < kMaxR; r++) m1[r] = m2[r] = A::zero();
                for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) {
                    Rv acc[kMaxR], u[kMaxR];
                    K::spmm_row(y, i, uj, acc);
                    K::ld_row(uj, i, R, u);
                    const Rv di = K::dinv_of(y, i);
#pragma unroll
                    for (int r = 0; r < kMaxR; r++) {
                        if (r >= R) continue;
                        A::st(au + (size_t)i * R + r, acc[r]);
                        m1[r] = A::fma(u[r], acc[r], m1[r]);
                        if (un || want_m2) {
                            const Rv z = A::mul(di, acc[r]);
                            if (un) A::st(un + (size_t)i * R + r, z);
                            m2[r] = A::fma(acc[r], z, m2[r]);
                        }
                    }
                }
                Rv v[2 * kMaxR];
                for (int r = 0; r < R; r++) {
                    v[r] = m1[r];
                    v[R + r] = m2[r];
                }
                const int nv = want_m2 ? 2 * R : R;
                double out = 0.0;
                cta_sum_n<A>(v, nv, red, &out);
                if (threadIdx.x < nv) {
                    const int q = threadIdx.x < R ? 2 * j : 2 * j + 1;  // moment slot: mu_{q+1}
                    const int r = threadIdx.x % R;
                    y.lpart[(size_t)(q * R + r) * y.items + li] = out;
                }
            }
            if (!grid_sync(a.g)) return;
        }

        // ------------------------------------------------------- solve
        for (int k = blockIdx.x; k < a.nsys; k += gridDim.x) {
            const BSys& y = a.sys[k];
            BCtl* bc = &a.bctl[k];
            const int state = bc->state;
            if (state == SYS_FINISHED) continue;
            const int R = y.R, items = y.items, step = bc->step;
            // rows to reduce: EXPORT: true residual (R); ACTIVE: ||r||^2, mu_0
            // (+ ||b||^2 at step 0) and the 2s-1 moments
            const int nu = state == SYS_EXPORT ? R : (step == 0 ? 3 * R : 2 * R);
            const int ubase = state == SYS_EXPORT ? 2 * R : 0;
            const int nl = state == SYS_EXPORT ? 0 : (2 * s - 1) * R;
            for (int q = warp; q < nu + nl; q += kBWarps) {
                const double* src = q < nu ? y.upart + (size_t)(ubase + q) * items
                                           : y.lpart + (size_t)(q - nu) * items;
                double t = 0.0;
                for (int b = lane; b < items; b += 32) t += __ldcg(src + b);
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
                if (lane == 0) sw_red[q] = t;
            }
            __syncthreads();
            if (state == SYS_EXPORT) {
                if (threadIdx.x < R) {
                    Ctrl* c = &a.rc[y.rhs0 + threadIdx.x];
                    c->true_res2 = sw_red[threadIdx.x];
                }
                if (threadIdx.x == 0) {
                    bc->state = SYS_FINISHED;
                    bc->t_fin = globaltimer();
                    atomicAdd(&a.g->finished, 1);
                }
                __syncthreads();
                continue;
            }
            if (warp < R) {
                Ctrl* c = &a.rc[y.rhs0 + warp];
                int decided = 0;
                if (lane == 0 && !c->done) {
                    if (step == 0) {
                        c->bnorm = sqrt(sw_red[2 * R + warp]);
                        if (c->bnorm == 0.0) {
                            c->zero_rhs = 1;
                            c->relres = 0.0;
                            c->status = 0;
                            c->step = 0;
                            c->done = 1;
                            decided = 1;
                        }
                    }
                    if (!decided) {
                        const double rel = sqrt(sw_red[warp]) / c->bnorm;
                        c->relres = rel;
                        c->step = step;
                        if (!isfinite(rel)) {
                            c->status = SSCG_BREAKDOWN;
                            c->done = 1;
                        } else if (rel < a.tol) {
                            c->status = 0;
                            c->done = 1;
                        } else if (step >= a.maxit) {
                            c->status = SSCG_NOT_CONVERGED;
                            c->done = 1;
                        }
                    }
                    if (!c->done) {
                        c->mu[0] = sw_red[R + warp];
                        for (int q = 0; q < 2 * s - 1; q++) c->mu[q + 1] = sw_red[nu + q * R + warp];
                    }
                }
                __syncwarp();
                const int run = __shfl_sync(0xffffffffu, c->done ? 0 : 1, 0);
                if (run) {
                    const int st = warp_sw_monomial(c, s, step, &scratch[warp]);
                    if (lane == 0 && st != 0) {
                        c->status = SSCG_BREAKDOWN;
                        c->done = 1;
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int all = 1;
                for (int r = 0; r < R; r++) all &= a.rc[y.rhs0 + r].done ? 1 : 0;
                if (all) bc->state = SYS_EXPORT;
                else bc->step = step + 1;
            }
            __syncthreads();
        }
        if (!grid_sync(a.g)) return;
        if (*(volatile int*)&a.g->finished >= a.nsys) break;

        // ------------------------------------------------------ update
        for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
            const int k = __ldg(a.item_sys + it);
            const BSys& y = a.sys[k];
            const int state = __ldcg(&a.bctl[k].state);
            if (state == SYS_FINISHED) continue;
            const int li = it - y.item0, R = y.R;
            const int r0 = li * y.T, r1 = min(y.n, r0 + y.T);
            if (state == SYS_EXPORT) {
                if (a.tuning) continue;
                double* X = const_cast<double*>(a.io[2 * k + 1]);
                const S* xw = reinterpret_cast<const S*>(y.xw);
                for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) {
#pragma unroll
                    for (int r = 0; r < kMaxR; r++) {
                        if (r >= R) continue;
                        const Ctrl* c = &a.rc[y.rhs0 + r];
                        double* px = X + (size_t)r * y.n + i;
                        *px = __ldcg(&c->zero_rhs) ? 0.0 : *px + A::to_d(A::ldcg(xw + (size_t)i * R + r));
                    }
                }
                continue;
            }
            const int kk = __ldcg(&a.bctl[k].step) - 1;  // the outer step being completed
            __syncthreads();
            for (int e = threadIdx.x; e < R * (s + s * s + 1); e += kBThreads) {
                const int r = e / (s + s * s + 1), q = e % (s + s * s + 1);
                const Ctrl* c = &a.rc[y.rhs0 + r];
                if (q < s) s_alpha[r][q] = __ldcg(c->alpha + q);
                else if (q < s + s * s) s_beta[r][q - s] = __ldcg(c->beta + (q - s));
                else s_act[r] = __ldcg(&c->done) ? 0 : 1;
            }
            __syncthreads();
            S* nb = reinterpret_cast<S*>(y.blk[kk & 1]);
            S* ob = reinterpret_cast<S*>(y.blk[(kk + 1) & 1]);
            const size_t nR = (size_t)y.n * R;
            S* xw = reinterpret_cast<S*>(y.xw);
            S* rv = reinterpret_cast<S*>(y.r);
            Rv rr[kMaxR], rz[kMaxR];
#pragma unroll
            for (int r = 0; r < kMaxR; r++) rr[r] = rz[r] = A::zero();
            for (int i = r0 + threadIdx.x; i < r1; i += kBThreads) {
                const Rv di = K::dinv_of(y, i);
                for (int r = 0; r < R; r++) {
                    const size_t o = (size_t)i * R + r;
                    Rv res = A::ldcg(rv + o);
                    if (s_act[r]) {
                        Rv po[kMaxSB], apo[kMaxSB];
                        if (kk > 0) {
#pragma unroll
                            for (int l = 0; l < kMaxSB; l++)
                                if (l < s) {
                                    po[l] = A::ldcg(ob + l * nR + o);
                                    apo[l] = A::ldcg(ob + (s + l) * nR + o);
                                }
                        }
                        Rv x = A::ldcg(xw + o);
#pragma unroll
                        for (int jj = 0; jj < kMaxSB; jj++) {
                            if (jj >= s) continue;
                            Rv p = A::ldcg(nb + jj * nR + o);
                            Rv ap = A::ldcg(nb + (s + jj) * nR + o);
                            if (kk > 0) {
#pragma unroll
                                for (int l = 0; l < kMaxSB; l++)
                                    if (l < s) {
                                        const Rv bl = A::from_d(s_beta[r][l + jj * s]);
                                        p = A::fma(po[l], bl, p);
                                        ap = A::fma(apo[l], bl, ap);
                                    }
                                A::st(nb + jj * nR + o, p);
                                A::st(nb + (s + jj) * nR + o, ap);
                            }
                            const double al = s_alpha[r][jj];
                            x = A::fma(p, A::from_d(al), x);
                            res = A::fma(ap, A::from_d(-al), res);
                        }
                        A::st(xw + o, x);
                        A::st(rv + o, res);
                        rr[r] = A::fma(res, res, rr[r]);
                    }
                    const Rv z = A::mul(di, res);
                    A::st(ob + o, z);  // U_0 of the next step (P_old_0 already read)
                    if (s_act[r]) rz[r] = A::fma(res, z, rz[r]);
                }
            }
            Rv v[2 * kMaxR];
            for (int r = 0; r < R; r++) {
                v[r] = rr[r];
                v[R + r] = rz[r];
            }
            double out = 0.0;
            cta_sum_n<A>(v, 2 * R, red, &out);
            if (threadIdx.x < 2 * R) y.upart[(size_t)threadIdx.x * y.items + li] = out;
        }
        if (!grid_sync(a.g)) return;
    }
}

int size_class(int64_t n) {
    if (n < (1 << 16)) return 0;
    if (n < (1 << 19)) return 1;
    if (n < (1 << 21)) return 2;
    return 3;
}

constexpr int kDefaultTile[4] = {256, 1024, 2048, 4096};

}  // namespace

}  // namespace sscg

using namespace sscg;

struct sscg_batch {
    sscg_ctx* ctx;
    int nsys, s, arith, maxit, total_rhs, nitems, grid, graph_ok;
    double tol;
    std::vector<const sscg_mat*> mats;
    std::vector<int> R, T;
    std::vector<BSys> hsys;
    // device (inside the caller's workspace)
    BSys* d_sys;
    int* d_item_sys;
    GCtl* d_g;
    BCtl* d_bctl;
    Ctrl* d_rc;
    const double** d_io;
    // pinned host mirrors
    const double** h_io;
    Ctrl* h_rc;
    BCtl* h_bctl;
    GCtl* h_g;
    cudaGraphExec_t exec;
    float last_ms;
};

namespace {

struct BLayout {
    size_t bytes;
    std::vector<size_t> off_blk0, off_blk1, off_xw, off_r, off_l, off_u;
    size_t off_sys, off_items, off_g, off_bctl, off_rc, off_io;
};

size_t elem_bytes(int arith) { return arith == SSCG_ARITH_F64 ? sizeof(double) : sizeof(float2); }

BLayout batch_layout(int nsys, const sscg_mat* const* mats, const int* nrhs, int s, int arith) {
    BLayout L;
    Carve c(nullptr, 0);
    int64_t items = 0, rhs = 0;
    for (int k = 0; k < nsys; k++) {
        items += (mats[k]->n + kMinTile - 1) / kMinTile;
        rhs += nrhs[k];
    }
    L.off_g = c.used;
    c.take<GCtl>(1);
    L.off_bctl = c.used = align_up(c.used, 256);
    c.take<BCtl>(nsys);
    L.off_rc = c.used = align_up(c.used, 256);
    c.take<Ctrl>(rhs);
    L.off_sys = c.used = align_up(c.used, 256);
    c.take<BSys>(nsys);
    L.off_items = c.used = align_up(c.used, 256);
    c.take<int>(items);
    L.off_io = c.used = align_up(c.used, 256);
    c.take<const double*>(2 * (size_t)nsys);
    const size_t eb = elem_bytes(arith);
    for (int k = 0; k < nsys; k++) {
        const size_t nR = (size_t)mats[k]->n * nrhs[k];
        const size_t it = (mats[k]->n + kMinTile - 1) / kMinTile;
        auto take = [&](size_t bytes) {
            c.used = align_up(c.used, 256);
            size_t o = c.used;
            c.used += align_up(bytes, 256);
            return o;
        };
        L.off_blk0.push_back(take(2 * (size_t)s * nR * eb));
        L.off_blk1.push_back(take(2 * (size_t)s * nR * eb));
        L.off_xw.push_back(take(nR * eb));
        L.off_r.push_back(take(nR * eb));
        L.off_l.push_back(take((size_t)(2 * s - 1) * nrhs[k] * it * sizeof(double)));
        L.off_u.push_back(take((size_t)3 * nrhs[k] * it * sizeof(double)));
    }
    L.bytes = align_up(c.used, 256);
    return L;
}

int check_batch(sscg_ctx* ctx, int nsys, const sscg_mat* const* mats, const int* nrhs, const sscg_opts* o) {
    if (nsys < 1 || nsys > SSCG_BATCH_MAX_SYSTEMS || !mats || !nrhs || !o)
        return set_err(ctx, SSCG_ERR_INVALID, "batch of %d systems (1..%d) or null argument", nsys,
                       SSCG_BATCH_MAX_SYSTEMS);
    if (o->s < 1 || o->s > kMaxSB) return set_err(ctx, SSCG_ERR_INVALID, "batch s = %d outside 1..%d", o->s, kMaxSB);
    if (o->basis != SSCG_BASIS_MONOMIAL) return set_err(ctx, SSCG_ERR_INVALID, "batched solves use the monomial basis");
    if (o->arith != SSCG_ARITH_F64 && o->arith != SSCG_ARITH_DF64)
        return set_err(ctx, SSCG_ERR_INVALID, "batched solves run in f64 or df64 arithmetic");
    if (o->maxit < 0 || !(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad maxit or tol");
    for (int k = 0; k < nsys; k++) {
        if (!mats[k]) return set_err(ctx, SSCG_ERR_INVALID, "system %d: null matrix", k);
        if (nrhs[k] < 1 || nrhs[k] > kMaxR)
            return set_err(ctx, SSCG_ERR_INVALID, "system %d: %d right-hand sides (1..%d)", k, nrhs[k], kMaxR);
        if (mats[k]->prec != SSCG_PREC_JACOBI)
            return set_err(ctx, SSCG_ERR_INVALID, "system %d: batched solves use the Jacobi preconditioner", k);
        if ((int64_t)mats[k]->n * nrhs[k] * 2 * kMaxSB >= ((int64_t)1 << 40))
            return set_err(ctx, SSCG_ERR_INVALID, "system %d too large", k);
    }
    return SSCG_OK;
}

// Rebuild the item table for the current tiles and upload descriptors.
int upload_plan(sscg_batch* b) {
    std::vector<int> item_sys;
    for (int k = 0; k < b->nsys; k++) {
        BSys& y = b->hsys[k];
        y.T = b->T[k];
        y.items = (y.n + y.T - 1) / y.T;
        y.item0 = (int)item_sys.size();
        for (int i = 0; i < y.items; i++) item_sys.push_back(k);
    }
    b->nitems = (int)item_sys.size();
    sscg_ctx* ctx = b->ctx;
    SSCG_CUDA(ctx, cudaMemcpyAsync(b->d_sys, b->hsys.data(), sizeof(BSys) * b->nsys, cudaMemcpyHostToDevice,
                                   ctx->stream));
    SSCG_CUDA(ctx, cudaMemcpyAsync(b->d_item_sys, item_sys.data(), sizeof(int) * item_sys.size(),
                                   cudaMemcpyHostToDevice, ctx->stream));
    SSCG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SSCG_OK;
}

template <class A>
int launch_batch(sscg_batch* b, int tuning, int maxit) {
    BArgs a;
    a.nsys = b->nsys;
    a.nitems = b->nitems;
    a.s = b->s;
    a.maxit = maxit;
    a.tuning = tuning;
    a.tol = tuning ? 0.0 : b->tol;
    a.sys = b->d_sys;
    a.item_sys = b->d_item_sys;
    a.io = b->d_io;
    a.g = b->d_g;
    a.bctl = b->d_bctl;
    a.rc = b->d_rc;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    SSCG_CUDA(b->ctx, cudaLaunchKernelEx(&cfg, k_batch<A>, a));
    return SSCG_OK;
}

int launch_any(sscg_batch* b, int tuning, int maxit) {
    return b->arith == SSCG_ARITH_F64 ? launch_batch<ArithF64>(b, tuning, maxit)
                                      : launch_batch<ArithDF64>(b, tuning, maxit);
}

// Reset the per-solve state on the stream: control blocks zeroed.
int reset_state(sscg_batch* b) {
    sscg_ctx* ctx = b->ctx;
    SSCG_CUDA(ctx, cudaMemsetAsync(b->d_g, 0, sizeof(GCtl), ctx->stream));
    SSCG_CUDA(ctx, cudaMemsetAsync(b->d_bctl, 0, sizeof(BCtl) * b->nsys, ctx->stream));
    SSCG_CUDA(ctx, cudaMemsetAsync(b->d_rc, 0, sizeof(Ctrl) * b->total_rhs, ctx->stream));
    return SSCG_OK;
}

// Autotuner: for each size class present, time a few outer steps of that
// class's systems alone (synthetic right-hand sides) with every candidate
// tile and keep the fastest.
int autotune(sscg_batch* b) {
    sscg_ctx* ctx = b->ctx;
    cudaEvent_t e0, e1;
    SSCG_CUDA(ctx, cudaEventCreate(&e0));
    SSCG_CUDA(ctx, cudaEventCreate(&e1));
    const std::vector<BSys> all = b->hsys;
    const std::vector<int> allT = b->T;
    const int nsys = b->nsys;
    int rc = SSCG_OK;
    std::vector<int> best(4, 0);
    for (int cls = 0; cls < 4 && rc == SSCG_OK; cls++) {
        std::vector<int> members;
        for (int k = 0; k < nsys; k++)
            if (size_class(all[k].n) == cls) members.push_back(k);
        if (members.empty()) continue;
        float best_ms = 1e30f;
        for (int ci = 0; ci < kNumCand && rc == SSCG_OK; ci++) {
            // sub-batch: the class's systems only, packed at the front
            b->nsys = (int)members.size();
            b->hsys.clear();
            b->T.clear();
            for (int k : members) {
                b->hsys.push_back(all[k]);
                b->T.push_back(kTileCand[ci]);
            }
            if ((rc = upload_plan(b))) break;
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && rc == SSCG_OK; rep++) {
                if ((rc = reset_state(b))) break;
                cudaEventRecord(e0, ctx->stream);
                if ((rc = launch_any(b, 1, 2))) break;
                cudaEventRecord(e1, ctx->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = set_err(ctx, SSCG_ERR_CUDA, "autotune run failed: %s", cudaGetErrorString(cudaGetLastError()));
                    break;
                }
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                GCtl g;
                cudaMemcpy(&g, b->d_g, sizeof(g), cudaMemcpyDeviceToHost);
                if (g.err) rc = set_err(ctx, g.err, "autotune run stopped (status %d)", g.err);
                ms = std::min(ms, t);
            }
            if (rc == SSCG_OK && ms < best_ms) {
                best_ms = ms;
                best[cls] = kTileCand[ci];
            }
        }
    }
    b->nsys = nsys;
    b->hsys = all;
    b->T = allT;
    for (int k = 0; k < nsys; k++)
        if (best[size_class(all[k].n)]) b->T[k] = best[size_class(all[k].n)];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return upload_plan(b);
}

// Capture one solve (state reset, io table upload, kernel, results back) as
// a CUDA graph; on a capture failure the plan launches directly.
void build_graph(sscg_batch* b) {
    sscg_ctx* ctx = b->ctx;
    cudaStream_t st = ctx->stream;
    cudaGraph_t graph = nullptr;
    b->graph_ok = 0;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    bool ok = reset_state(b) == SSCG_OK;
    ok = ok && cudaMemcpyAsync(b->d_io, b->h_io, sizeof(double*) * 2 * b->nsys, cudaMemcpyHostToDevice, st) ==
                   cudaSuccess;
    ok = ok && launch_any(b, 0, b->maxit) == SSCG_OK;
    ok = ok && cudaMemcpyAsync(b->h_rc, b->d_rc, sizeof(Ctrl) * b->total_rhs, cudaMemcpyDeviceToHost, st) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(b->h_bctl, b->d_bctl, sizeof(BCtl) * b->nsys, cudaMemcpyDeviceToHost, st) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(b->h_g, b->d_g, sizeof(GCtl), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (!ok || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return;
    }
    if (cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess) b->graph_ok = 1;
    else b->exec = nullptr;
    cudaGraphDestroy(graph);
    cudaGetLastError();
}

}  // namespace

extern "C" {

int sscg_batch_workspace_bytes(int nsys, const sscg_mat* const* mats, const int* nrhs, const sscg_opts* opts,
                               size_t* bytes) {
    if (!bytes) return SSCG_ERR_INVALID;
    if (check_batch(nullptr, nsys, mats, nrhs, opts)) return SSCG_ERR_INVALID;
    *bytes = batch_layout(nsys, mats, nrhs, opts->s, opts->arith).bytes;
    return SSCG_OK;
}

int sscg_batch_create(sscg_ctx* ctx, int nsys, const sscg_mat* const* mats, const int* nrhs, const sscg_opts* opts,
                      int tune, void* ws, size_t ws_bytes, sscg_batch** out) {
    if (!ctx || !out) return SSCG_ERR_INVALID;
    if (int e = check_batch(ctx, nsys, mats, nrhs, opts)) return e;
    const BLayout L = batch_layout(nsys, mats, nrhs, opts->s, opts->arith);
    if (!ws || ws_bytes < L.bytes || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", L.bytes,
                       ws_bytes);
    sscg_batch* b = new sscg_batch();
    b->ctx = ctx;
    b->nsys = nsys;
    b->s = opts->s;
    b->arith = opts->arith;
    b->maxit = opts->maxit;
    b->tol = opts->tol;
    char* base = (char*)ws;
    b->d_g = (GCtl*)(base + L.off_g);
    b->d_bctl = (BCtl*)(base + L.off_bctl);
    b->d_rc = (Ctrl*)(base + L.off_rc);
    b->d_sys = (BSys*)(base + L.off_sys);
    b->d_item_sys = (int*)(base + L.off_items);
    b->d_io = (const double**)(base + L.off_io);
    int rhs = 0;
    for (int k = 0; k < nsys; k++) {
        const sscg_mat* m = mats[k];
        BSys y;
        memset(&y, 0, sizeof(y));
        y.rowptr = m->rowptr;
        y.col = m->col;
        y.val = m->val;
        y.vhi = m->vhi;
        y.vlo = m->vlo;
        y.dinv = opts->arith == SSCG_ARITH_F64 ? (const void*)m->dinv : (const void*)m->dinv_df;
        y.blk[0] = base + L.off_blk0[k];
        y.blk[1] = base + L.off_blk1[k];
        y.xw = base + L.off_xw[k];
        y.r = base + L.off_r[k];
        y.lpart = (double*)(base + L.off_l[k]);
        y.upart = (double*)(base + L.off_u[k]);
        y.n = (int)m->n;
        y.R = nrhs[k];
        y.exact = m->exact_fp32;
        y.rhs0 = rhs;
        rhs += nrhs[k];
        b->mats.push_back(m);
        b->R.push_back(nrhs[k]);
        b->T.push_back(kDefaultTile[size_class(m->n)]);
        b->hsys.push_back(y);
    }
    b->total_rhs = rhs;
    auto fail = [&](int rc) {
        sscg_batch_destroy(b);
        return rc;
    };
    int per_sm = 0;
    cudaError_t e = opts->arith == SSCG_ARITH_F64
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<ArithF64>, kBThreads, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<ArithDF64>, kBThreads, 0);
    if (e != cudaSuccess || per_sm < 1)
        return fail(set_err(ctx, SSCG_ERR_CUDA, "batched kernel cannot be resident: %s", cudaGetErrorString(e)));
    b->grid = per_sm * ctx->sm_count;
    if (cudaMallocHost((void**)&b->h_io, sizeof(double*) * 2 * nsys) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_rc, sizeof(Ctrl) * rhs) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_bctl, sizeof(BCtl) * nsys) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_g, sizeof(GCtl)) != cudaSuccess)
        return fail(set_err(ctx, SSCG_ERR_CUDA, "pinned host buffers"));
    memset(b->h_io, 0, sizeof(double*) * 2 * nsys);
    if (int rc = upload_plan(b)) return fail(rc);
    if (tune)
        if (int rc = autotune(b)) return fail(rc);
    build_graph(b);
    *out = b;
    return SSCG_OK;
}

int sscg_batch_destroy(sscg_batch* b) {
    if (!b) return SSCG_ERR_INVALID;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->h_io) cudaFreeHost(b->h_io);
    if (b->h_rc) cudaFreeHost(b->h_rc);
    if (b->h_bctl) cudaFreeHost(b->h_bctl);
    if (b->h_g) cudaFreeHost(b->h_g);
    delete b;
    return SSCG_OK;
}

int sscg_batch_solve(sscg_batch* b, const double* const* B, double* const* X, sscg_info* infos,
                     sscg_info* rhs_infos, double* latency_ms) {
    if (!b) return SSCG_ERR_INVALID;
    sscg_ctx* ctx = b->ctx;
    if (!B || !X) return set_err(ctx, SSCG_ERR_INVALID, "null B or X table");
    for (int k = 0; k < b->nsys; k++) {
        if (!B[k] || !X[k]) return set_err(ctx, SSCG_ERR_INVALID, "system %d: null B or X", k);
        b->h_io[2 * k] = B[k];
        b->h_io[2 * k + 1] = X[k];
    }
    cudaStream_t st = ctx->stream;
    cudaEvent_t e0, e1;
    SSCG_CUDA(ctx, cudaEventCreate(&e0));
    SSCG_CUDA(ctx, cudaEventCreate(&e1));
    SSCG_CUDA(ctx, cudaEventRecord(e0, st));
    if (b->graph_ok) {
        SSCG_CUDA(ctx, cudaGraphLaunch(b->exec, st));
    } else {
        if (int rc = reset_state(b)) return rc;
        SSCG_CUDA(ctx, cudaMemcpyAsync(b->d_io, b->h_io, sizeof(double*) * 2 * b->nsys, cudaMemcpyHostToDevice, st));
        if (int rc = launch_any(b, 0, b->maxit)) return rc;
        SSCG_CUDA(ctx, cudaMemcpyAsync(b->h_rc, b->d_rc, sizeof(Ctrl) * b->total_rhs, cudaMemcpyDeviceToHost, st));
        SSCG_CUDA(ctx, cudaMemcpyAsync(b->h_bctl, b->d_bctl, sizeof(BCtl) * b->nsys, cudaMemcpyDeviceToHost, st));
        SSCG_CUDA(ctx, cudaMemcpyAsync(b->h_g, b->d_g, sizeof(GCtl), cudaMemcpyDeviceToHost, st));
    }
    SSCG_CUDA(ctx, cudaEventRecord(e1, st));
    SSCG_CUDA(ctx, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->last_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const GCtl& g = *b->h_g;
    if (g.err) return set_err(ctx, g.err, "batched solve stopped: a grid barrier wait expired");
    int worst = SSCG_OK;
    for (int k = 0; k < b->nsys; k++) {
        const BSys& y = b->hsys[k];
        int st_k = SSCG_OK, it = 0;
        double rr = 0.0, rt = 0.0;
        for (int r = 0; r < y.R; r++) {
            const Ctrl& c = b->h_rc[y.rhs0 + r];
            const double rel_true = c.zero_rhs ? 0.0 : sqrt(c.true_res2) / c.bnorm;
            if (c.status == SSCG_BREAKDOWN) st_k = SSCG_BREAKDOWN;
            else if (c.status == SSCG_NOT_CONVERGED && st_k == SSCG_OK) st_k = SSCG_NOT_CONVERGED;
            it = std::max(it, c.step);
            rr = std::max(rr, c.relres);
            rt = std::max(rt, rel_true);
            if (rhs_infos) {
                sscg_info& ri = rhs_infos[y.rhs0 + r];
                ri.status = c.status;
                ri.outer_iters = c.step;
                ri.equiv_iters = (int64_t)c.step * b->s;
                ri.rel_res_recursive = c.relres;
                ri.rel_res_true = rel_true;
                ri.hist_len = 0;
            }
        }
        if (infos) {
            sscg_info& in = infos[k];
            in.status = st_k;
            in.outer_iters = it;
            in.equiv_iters = (int64_t)it * b->s;
            in.rel_res_recursive = rr;
            in.rel_res_true = rt;
            in.hist_len = 0;
            in.kernel_launches = 1;
        }
        if (latency_ms) latency_ms[k] = (double)(b->h_bctl[k].t_fin - g.t0) * 1e-6;
        if (st_k > worst) worst = st_k;
    }
    return worst;
}

int sscg_batch_props(const sscg_batch* b, int* tile_rows, int* grid, int* graph, float* last_ms) {
    if (!b) return SSCG_ERR_INVALID;
    if (tile_rows)
        for (int k = 0; k < b->nsys; k++) tile_rows[k] = b->T[k];
    if (grid) *grid = b->grid;
    if (graph) *graph = b->graph_ok;
    if (last_ms) *last_ms = b->last_ms;
    return SSCG_OK;
}

}  // extern "C"
