// Preconditioned CG (Algorithm 1), the comparator of the s-step method, on
// the same SpMV tiles and arithmetic, and the Lanczos spectral-bound
// estimate built on it.  Per iteration:
//   k_pcg_spmv   : s_k = A p_k and p_k . s_k; last CTA forms alpha_k
//   k_pcg_update : x += alpha p, r -= alpha s, ||r||^2 (and, with a diagonal
//                  B, u = B^-1 r and u . r); last CTA tests convergence and,
//                  with a diagonal B, forms beta_k
//   (Chebyshev B: the preconditioner kernels, then k_pcg_rho for u . r, beta_k)
//   k_pcg_dir    : p_{k+1} = u_{k+1} + beta_k p_k
// The Lanczos estimate runs k steps from y = 0 on A y = r0 and takes the
// extreme Ritz values of B^-1 A from the CG coefficients:
//   T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T_{j,j+1} = sqrt(beta_j)/alpha_j
// (Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.7.3).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "prec.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

__device__ __forceinline__ int done_of(const Ctrl* c) { return __ldcg(&c->done); }

template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_pcg_init(MatView M, const typename A::S* __restrict__ dinv, int diag,
                                                       const double* __restrict__ b, const double* __restrict__ x0,
                                                       typename A::S* __restrict__ xw, typename A::S* __restrict__ r,
                                                       typename A::S* __restrict__ p, double* __restrict__ part,
                                                       Ctrl* ctrl, double* __restrict__ hist) {
    using R = typename A::R;
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    __shared__ double red[3 * (kThreads / 32)];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    R rr = A::zero(), ru = A::zero();
    double bb = 0.0, bmax = 0.0;  // ||b||^2 and max |b_i| in FP64 whatever the arithmetic
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        R y = A::zero();
        int row = tile * kTileRows + threadIdx.x;
        bool live = row < M.n;
        if (x0) live = tile_spmv<A, VM>(M, tile, [&](int c) { return A::from_d(__ldg(x0 + c)); }, y, row, smem, s_rp);
        if (live) {
            const double bd = b[row];
            R bi = A::from_d(bd);
            R ri = A::sub(bi, y);
            if (xw) A::st(xw + row, A::zero());  // DF64 iterate holds x - x0
            A::st(r + row, ri);
            bb = fma(bd, bd, bb);
            bmax = fmax(bmax, fabs(bd));
            rr = A::fma(ri, ri, rr);
            if (diag) {
                R ui = dinv ? A::mul(A::ld(dinv + row), ri) : ri;
                A::st(p + row, ui);
                ru = A::fma(ri, ui, ru);
            }
        }
    }
    R v[2] = {rr, ru};
    double out[2];
    block_sum<A, 2>(v, red, out);
    double vb[1] = {bb}, outb[1];
    block_sum<ArithF64, 1>(vb, red, outb);
    const double bm = block_max(isfinite(bmax) ? bmax : 0.0, red);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = outb[0];
        part[G + blockIdx.x] = out[0];
        part[2 * G + blockIdx.x] = out[1];
        part[3 * G + blockIdx.x] = bm;
    }
    if (!last_cta(&ctrl->ticket[0])) return;
    __shared__ double sh[32];
    double sbb = cta_sum_partials(part, G, sh);
    double srr = cta_sum_partials(part + G, G, sh);
    double sru = cta_sum_partials(part + 2 * G, G, sh);
    const double smax = cta_max_partials(part + 3 * G, G, sh);
    if (threadIdx.x == 0) {
        ctrl->bnorm = sqrt(sbb);
        ctrl->rho = sru;
        ctrl->nhist = 1;
        if (A::kind != 0 && isfinite(sbb) && sbb != 0.0 && (smax < kDfRhsMin || smax > kDfRhsMax)) {
            ctrl->status = SSCG_ERR_INVALID;
            ctrl->done = 1;
        } else if (sbb == 0.0) {
            ctrl->zero_rhs = 1;
            ctrl->relres = 0.0;
            hist[0] = 0.0;
            ctrl->status = 0;
            ctrl->done = 1;
        } else {
            double rel = sqrt(srr) / ctrl->bnorm;
            ctrl->relres = rel;
            hist[0] = rel;
            if (!isfinite(rel)) {
                ctrl->status = SSCG_ERR_NONFINITE;
                ctrl->done = 1;
            } else if (rel < ctrl->tol) {
                ctrl->status = 0;
                ctrl->done = 1;
            } else if (ctrl->maxit == 0) {
                ctrl->status = 1;
                ctrl->done = 1;
            }
        }
    }
}

// PCG's FP64 7-point SpMV measured fastest at 5 CTAs per SM (48 registers;
// the s-step level, with its second moment, at 4).
template <class A, int DM>
__host__ __device__ constexpr int pcg_spmv_min_blocks() {
    return (A::kind == 0 && DM == 7) ? 5 : dia_min_blocks<A, DM>();
}

template <class A, int VM, int DM>
__global__ void __launch_bounds__(kThreads, pcg_spmv_min_blocks<A, DM>()) k_pcg_spmv(MatView M, const typename A::S* __restrict__ p,
                                                       typename A::S* __restrict__ q, double* __restrict__ part,
                                                       Ctrl* ctrl) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    __shared__ double red[kThreads / 32];
    R pq = A::zero();
    auto xf = [&](int c) { return A::ldg(p + c); };
    auto epi = [&](int row, R y) {
        A::st(q + row, y);
        pq = A::fma(A::ldg(p + row), y, pq);
    };
    bool ok = true;
    if constexpr (DM >= 7 && A::kind == 0) {
        // FP64 diagonal form, Laplacian class: q = c_centre p + c_off S, one
        // FMA beyond the neighbour sum when c_off = -1 (the Poisson stencils)
        const double cc = M.dc[DM / 2], co = (double)M.dco;
        double a = 0.0;
        auto run = [&](auto qf) {
            spmv_dia_lap_f64<DM>(M, p, [&](int i, double S, double pc) {
                const double y = qf(S, pc);
                q[i] = y;
                a = fma(pc, y, a);
            });
        };
        if (co == -1.0) run([&](double S, double pc) { return fma(cc, pc, -S); });
        else run([&](double S, double pc) { return fma(co, S, cc * pc); });
        pq = a;
    } else if constexpr (DM != 0 && A::kind == 1) {
        DotAcc d{0.f, 0.f};
        spmv_dia_df<DM>(M, p, [&](int i, df64 y0, df64 x0, df64 y1, df64 x1, bool has1) {
            if (has1) st_pair(q + i, y0, y1);
            else A::st(q + i, y0);
            dot_add(d, x0, y0);
            dot_add(d, x1, y1);
            dot_renorm(d);
        });
        pq = dot_value(d);
    } else if constexpr (DM != 0) {
        spmv_dia<A>(M, xf, epi);
    } else {
        ok = spmv_pipe<A, VM, kStages>(M, smem, xf, epi, ctrl);
    }
    if (!ok) return;
    R v[1] = {pq};
    double out[1];
    block_sum<A, 1>(v, red, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
    if (!last_cta(&ctrl->ticket[1])) return;
    __shared__ double sh[32];
    double t = cta_sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
        if (!(t > 0.0) || !isfinite(t) || !isfinite(ctrl->rho)) {
            ctrl->status = 2;
            ctrl->done = 1;
        } else {
            ctrl->pcg_alpha = ctrl->rho / t;
        }
    }
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_pcg_update(int n, int diag, typename A::S* __restrict__ x,
                                                         typename A::S* __restrict__ r,
                                                         const typename A::S* __restrict__ p,
                                                         const typename A::S* __restrict__ q,
                                                         const typename A::S* __restrict__ dinv, double dinv_c,
                                                         double* __restrict__ part, Ctrl* ctrl,
                                                         double* __restrict__ hist, double* __restrict__ coef) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    __shared__ double red[2 * (kThreads / 32)];
    const R alpha = A::from_d(ctrl->pcg_alpha), nalpha = A::from_d(-ctrl->pcg_alpha);
    const R dc = A::from_d(dinv_c);
    R rr = A::zero(), ru = A::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R pi = A::ld(p + i);
        R xi = A::fma(alpha, pi, A::ld(x + i));
        R ri = A::fma(nalpha, A::ld(q + i), A::ld(r + i));
        A::st(x + i, xi);
        A::st(r + i, ri);
        rr = A::fma(ri, ri, rr);
        if (diag && dinv) ru = A::fma(ri, A::mul(A::ld(dinv + i), ri), ru);
    }
    // u = B^-1 r with B^-1 the constant dinv_c (or the identity): u . r = dinv_c ||r||^2
    if (diag && !dinv) ru = dinv_c != 0.0 ? A::mul(dc, rr) : rr;
    R v[2] = {rr, ru};
    double out[2];
    block_sum<A, 2>(v, red, out);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = out[0];
        part[G + blockIdx.x] = out[1];
    }
    if (!last_cta(&ctrl->ticket[2])) return;
    __shared__ double sh[32];
    double srr = cta_sum_partials(part, G, sh);
    double sru = cta_sum_partials(part + G, G, sh);
    if (threadIdx.x == 0) {
        int step = ctrl->step + 1;
        double rel = sqrt(srr) / ctrl->bnorm;
        if (coef) coef[2 * (step - 1)] = ctrl->pcg_alpha;
        if (diag) {
            ctrl->pcg_beta = sru / ctrl->rho;
            ctrl->rho = sru;
            if (coef) coef[2 * (step - 1) + 1] = ctrl->pcg_beta;
        }
        ctrl->step = step;
        ctrl->relres = rel;
        hist[step] = rel;
        ctrl->nhist = step + 1;
        if (!isfinite(rel)) {
            ctrl->status = 2;
            ctrl->done = 1;
        } else if (rel < ctrl->tol) {
            ctrl->status = 0;
            ctrl->done = 1;
        } else if (step >= ctrl->maxit) {
            ctrl->status = 1;
            ctrl->done = 1;
        }
    }
}

// rho = r . u with u = B^-1 r from the preconditioner kernels.  first: set
// rho; otherwise beta_k = rho_new / rho (recorded in coef).
template <class A>
__global__ void __launch_bounds__(kThreads) k_pcg_rho(int n, const typename A::S* __restrict__ r,
                                                      const typename A::S* __restrict__ u, int first,
                                                      double* __restrict__ part, Ctrl* ctrl,
                                                      double* __restrict__ coef) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    __shared__ double red[kThreads / 32];
    R ru = A::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        ru = A::fma(A::ld(r + i), A::ld(u + i), ru);
    R v[1] = {ru};
    double out[1];
    block_sum<A, 1>(v, red, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
    if (!last_cta(&ctrl->ticket[3])) return;
    __shared__ double sh[32];
    double t = cta_sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) {
        if (first) {
            ctrl->rho = t;
        } else {
            ctrl->pcg_beta = t / ctrl->rho;
            ctrl->rho = t;
            if (coef) coef[2 * (ctrl->step - 1) + 1] = ctrl->pcg_beta;
        }
        if (!(t > 0.0) || !isfinite(t)) {
            ctrl->status = 2;
            ctrl->done = 1;
        }
    }
}

template <class A>
__global__ void __launch_bounds__(kThreads) k_pcg_dir(int n, int diag, typename A::S* __restrict__ p,
                                                      const typename A::S* __restrict__ r,
                                                      const typename A::S* __restrict__ u,
                                                      const typename A::S* __restrict__ dinv, double dinv_c,
                                                      const Ctrl* ctrl) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    const R beta = A::from_d(ctrl->pcg_beta);
    const R dc = A::from_d(dinv_c);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R ui;
        if (diag) {
            R ri = A::ld(r + i);
            ui = dinv ? A::mul(A::ld(dinv + i), ri) : (dinv_c != 0.0 ? A::mul(dc, ri) : ri);
        } else {
            ui = A::ld(u + i);
        }
        A::st(p + i, A::fma(beta, A::ld(p + i), ui));
    }
}

// x = x0 + (x - x0) for DF64 (the iterate holds the correction); b = 0 gives 0.
template <class A>
__global__ void k_pcg_export(int n, const typename A::S* __restrict__ xw, double* __restrict__ x, const Ctrl* ctrl) {
    const int zero = ctrl->zero_rhs;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (zero) x[i] = 0.0;
        else if (A::kind != 0) x[i] = x[i] + A::to_d(A::ld(xw + i));
    }
}

__global__ void __launch_bounds__(kThreads) k_pcg_true_res(MatView M, const double* __restrict__ b,
                                                           const double* __restrict__ x, double* __restrict__ part,
                                                           Ctrl* ctrl) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    __shared__ double red[kThreads / 32];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    double acc = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        double y;
        int row;
        bool live = tile_spmv<ArithF64, VAL_F64>(M, tile, [&](int c) { return __ldg(x + c); }, y, row, smem, s_rp);
        if (live) {
            double t = b[row] - y;
            acc = fma(t, t, acc);
        }
    }
    double v[1] = {acc}, out[1];
    block_sum<ArithF64, 1>(v, red, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
    if (!last_cta(&ctrl->ticket[3])) return;
    __shared__ double sh[32];
    double t = cta_sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) ctrl->true_res2 = t;
}

// splitmix64 in counter form: draw i of the generator started at `seed` is
// mix(seed + (i+1) * 0x9E3779B97F4A7C15); U[-1,1) = 2 (z >> 11) 2^-53 - 1.
__global__ void k_splitmix_uniform(int n, unsigned long long seed, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[i] = (double)(z >> 11) * 0x1p-52 - 1.0;
    }
}

// Number of eigenvalues of the tridiagonal (d, e) below x (Sturm count).
__device__ int sturm_count(int k, const double* d, const double* e, double x) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0.0) cnt++;
    for (int i = 1; i < k; i++) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

// Extreme Ritz values from k CG steps (coef: alpha_j, beta_j pairs) by
// bisection on the Sturm count of the Lanczos tridiagonal (one thread).
__global__ void k_ritz(const double* __restrict__ coef, int k, double* __restrict__ dwork, Ctrl* ctrl) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* d = dwork;
    double* e = dwork + k;
    for (int j = 0; j < k; j++) {
        double a = coef[2 * j];
        d[j] = 1.0 / a + (j > 0 ? coef[2 * (j - 1) + 1] / coef[2 * (j - 1)] : 0.0);
        if (j + 1 < k) e[j] = sqrt(coef[2 * j + 1]) / a;
    }
    double lo = d[0], hi = d[0];
    for (int i = 0; i < k; i++) {
        double rad = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < k ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - rad);
        hi = fmax(hi, d[i] + rad);
    }
    double span = hi - lo + 1e-300;
    lo -= 1e-12 * span;
    hi += 1e-12 * span;
    for (int which = 0; which < 2; which++) {
        int target = which == 0 ? 1 : k;
        double l = lo, h = hi;
        for (int it = 0; it < 200 && h - l > 1e-15 * (fabs(l) + fabs(h)); it++) {
            double mid = 0.5 * (l + h);
            if (sturm_count(k, d, e, mid) >= target) h = mid;
            else l = mid;
        }
        ctrl->scratch[which] = 0.5 * (l + h);
    }
}

struct PLayout {
    Ctrl* ctrl;
    double* hist;
    double* part;
    double* coef;
    void *x, *r, *p, *q, *u, *tmp;
    double *bdev, *xdev;
    size_t bytes;
};

PLayout pplan(const sscg_mat* mat, int maxit, unsigned flags, void* base, size_t cap) {
    PLayout L{};
    size_t ldn = align_up((size_t)mat->n, 64);
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)maxit + 2);
    L.part = c.take<double>((size_t)8 * 160 * 4);
    L.coef = c.take<double>(2 * ((size_t)maxit + 2));
    L.x = c.take<double>(ldn);
    L.r = c.take<double>(ldn);
    // margins around p: the diagonal-form SpMV gathers it without clamping
    const size_t g = dia_margin(mat);
    if (g) c.take<double>(g);
    L.p = c.take<double>(ldn);
    if (g) c.take<double>(g);
    L.q = c.take<double>(ldn);
    if (mat->prec == SSCG_PREC_CHEB) {
        L.u = c.take<double>(ldn);
        L.tmp = c.take<double>(3 * ldn);
    }
    if (flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>(ldn);
        L.xdev = c.take<double>(ldn);
    }
    L.bytes = c.used;
    return L;
}

// One PCG run.  x may be null (zero start and no export; the Lanczos
// estimate); coef receives alpha_j, beta_j when not null.
template <class A, int VM, int DM>
int run_pcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, int maxit, const PLayout& L,
            const typename A::S* dinv, Ctrl* h, Prof& P, double* coef) {
    using S = typename A::S;
    constexpr bool DIA = DM != 0;
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n;
    const MatView M = mat_view(mat);
    const size_t smem = stage_bytes<A, VM>(M.cap), smem64 = stage_bytes<ArithF64, VAL_F64>(M.cap);
    const size_t smem_pipe = pipe_bytes<VM, kStages>(M.cap) + 128;
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pcg_init<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const size_t smem_sp = DIA ? 128 : smem_pipe;
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pcg_spmv<A, VM, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_sp));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_cheb_step<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pipe));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pcg_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    const int Gi = occupancy_grid(ctx, k_pcg_init<A, VM>, smem, n);
    const int Gs = occupancy_grid(ctx, k_pcg_spmv<A, VM, DM>, smem_sp, n);
    const int Gc = occupancy_grid(ctx, k_cheb_step<A, VM>, smem_pipe, n);
    const int Gu = occupancy_grid(ctx, k_pcg_update<A>, 0, n);
    const int Gd = occupancy_grid(ctx, k_pcg_dir<A>, 0, n);
    const int Gr = occupancy_grid(ctx, k_pcg_rho<A>, 0, n);
    const int Gt = occupancy_grid(ctx, k_pcg_true_res, smem64, n);
    const bool diag = mat->prec != SSCG_PREC_CHEB;
    // with the diagonal form, a Jacobi D is the constant diagonal value
    const bool cd = DIA && dinv != nullptr && diag;
    const typename A::S* dinv_it = cd ? nullptr : dinv;
    const double dinv_c = cd ? mat->dia_dinv : 0.0;
    ChebPrec<A, VM> cheb(diag ? 1 : mat->degree, diag ? 1.0 : mat->plmin, diag ? 2.0 : mat->plmax);
    const size_t ld = align_up((size_t)mat->n, 64);
    S* xw = (A::kind == 0) ? (S*)x : (S*)L.x;
    S* r = (S*)L.r;
    S* p = (S*)L.p;
    S* q = (S*)L.q;
    S* u = (S*)L.u;
    S* tmp = (S*)L.tmp;
    if (!x) xw = (S*)L.x;  // zero start: the iterate lives in the workspace
    P.begin();
    k_pcg_init<A, VM><<<Gi, kThreads, smem, st>>>(M, dinv, diag ? 1 : 0, b, x, (A::kind == 0 && x) ? nullptr : xw,
                                                  r, p, L.part, L.ctrl, L.hist);
    if (!diag) {
        P.launches += cheb.apply(M, dinv, r, p, tmp, ld, Gd, Gc, smem_pipe, st, L.ctrl);
        k_pcg_rho<A><<<Gr, kThreads, 0, st>>>(n, r, p, 1, L.part, L.ctrl, coef);
        P.launches++;
    }
    P.end(FAM_INIT, 0);
    SSCG_CUDA(ctx, cudaGetLastError());
    const int per_chunk = 16;
    ChunkPoll poll;
    SSCG_CUDA(ctx, poll.init());
    int launched = 0, err = 0;
    while (launched < maxit) {
        int c = std::min(per_chunk, maxit - launched);
        for (int k = 0; k < c; k++) {
            const int it = launched + k;
            P.begin();
            k_pcg_spmv<A, VM, DM><<<Gs, kThreads, smem_sp, st>>>(M, p, q, L.part, L.ctrl);
            P.end(FAM_MPK, it);
            P.begin();
            k_pcg_update<A><<<Gu, kThreads, 0, st>>>(n, diag ? 1 : 0, xw, r, p, q, dinv_it, dinv_c, L.part, L.ctrl,
                                                     L.hist, coef);
            P.end(FAM_UPDATE, it);
            P.begin();
            if (!diag) {
                P.launches += cheb.apply(M, dinv, r, u, tmp, ld, Gd, Gc, smem_pipe, st, L.ctrl);
                k_pcg_rho<A><<<Gr, kThreads, 0, st>>>(n, r, u, 0, L.part, L.ctrl, coef);
                P.launches++;
            }
            k_pcg_dir<A><<<Gd, kThreads, 0, st>>>(n, diag ? 1 : 0, p, r, u, dinv_it, dinv_c, L.ctrl);
            P.end(FAM_DIR, it);
        }
        if (cudaGetLastError() != cudaSuccess) {
            err = 1;
            break;
        }
        launched += c;
        int fin = 0;
        cudaError_t pe = cudaSuccess;
        const bool got = poll.step(ctx->pinned, &L.ctrl->done, st, &fin, &pe);
        SSCG_CUDA(ctx, pe);
        if (got && fin) break;
    }
    if (err) return set_err(ctx, SSCG_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (x) {
        P.begin();
        k_pcg_export<A><<<Gd, kThreads, 0, st>>>(n, xw, x, L.ctrl);
        k_pcg_true_res<<<Gt, kThreads, smem64, st>>>(M, b, x, L.part, L.ctrl);
        P.end(FAM_FINAL, 0);
        P.launches++;
    }
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(h, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return 0;
}

int dispatch_pcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, int maxit, int arith,
                 const PLayout& L, Ctrl* h, Prof& P, double* coef) {
    const bool scale = mat->prec != SSCG_PREC_NONE;  // Jacobi and Chebyshev scale by D^-1
    // the diagonal form serves the SpMV of a diagonal preconditioner (the
    // Chebyshev preconditioner's steps stage CSR tiles)
    const bool dia = mat->dia && mat->prec != SSCG_PREC_CHEB;
    if (arith == SSCG_ARITH_F64) {
        const double* d = scale ? mat->dinv : nullptr;
        // every PCG layout carves margins around p, the only vector the SpMV gathers
        const int dm = dia ? dia_mode(mat, true) : 0;
        if (dm == 7) return run_pcg<ArithF64, VAL_F64, 7>(ctx, mat, b, x, maxit, L, d, h, P, coef);
        if (dm == 27) return run_pcg<ArithF64, VAL_F64, 27>(ctx, mat, b, x, maxit, L, d, h, P, coef);
        if (dm != 0) return run_pcg<ArithF64, VAL_F64, 1>(ctx, mat, b, x, maxit, L, d, h, P, coef);
        return run_pcg<ArithF64, VAL_F64, 0>(ctx, mat, b, x, maxit, L, d, h, P, coef);
    }
    const float2* d = scale ? mat->dinv_df : nullptr;
    // every PCG layout carves margins around p, the only vector the SpMV gathers
    const int dm = dia ? dia_mode(mat, true) : 0;
    if (dm == 7) return run_pcg<ArithDF64, VAL_F32, 7>(ctx, mat, b, x, maxit, L, d, h, P, coef);
    if (dm == 27) return run_pcg<ArithDF64, VAL_F32, 27>(ctx, mat, b, x, maxit, L, d, h, P, coef);
    if (dm != 0) return run_pcg<ArithDF64, VAL_F32, 2>(ctx, mat, b, x, maxit, L, d, h, P, coef);
    if (mat->exact_fp32) return run_pcg<ArithDF64, VAL_F32, 0>(ctx, mat, b, x, maxit, L, d, h, P, coef);
    return run_pcg<ArithDF64, VAL_DF, 0>(ctx, mat, b, x, maxit, L, d, h, P, coef);
}

Ctrl fresh_ctrl(int maxit, double tol) {
    Ctrl h;
    memset(&h, 0, sizeof(h));
    h.status = 1;
    h.maxit = maxit;
    h.s = 1;
    h.tol = tol;
    return h;
}

}  // namespace

int pcg_workspace(const sscg_mat* mat, const sscg_opts* o, size_t* bytes) {
    *bytes = pplan(mat, o->maxit, o->flags, nullptr, 0).bytes;
    return 0;
}

int bounds_workspace(const sscg_mat* mat, int steps, size_t* bytes) {
    Carve c(nullptr, 0);
    c.used = pplan(mat, steps, 0, nullptr, 0).bytes;
    c.take<double>(align_up((size_t)mat->n, 64));  // r0
    c.take<double>(2 * (size_t)steps + 2);        // Ritz work
    *bytes = c.used;
    return 0;
}

int solve_pcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
              sscg_info* info, void* ws, size_t ws_bytes) {
    if (!mat || !o || !b || !x) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    if (o->maxit < 0 || !(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad maxit or tol");
    if (o->arith != SSCG_ARITH_F64 && o->arith != SSCG_ARITH_DF64)
        return set_err(ctx, SSCG_ERR_INVALID, "arith %d not supported by PCG", o->arith);
    size_t need = 0;
    pcg_workspace(mat, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    PLayout L = pplan(mat, o->maxit, o->flags, ws, ws_bytes);
    cudaStream_t st = ctx->stream;
    const int64_t n = mat->n;
    const double* bd = b;
    double* xd = x;
    if (o->flags & SSCG_HOST_VECTORS) {
        SSCG_CUDA(ctx, cudaMemcpyAsync(L.bdev, b, n * sizeof(double), cudaMemcpyHostToDevice, st));
        SSCG_CUDA(ctx, cudaMemcpyAsync(L.xdev, x, n * sizeof(double), cudaMemcpyHostToDevice, st));
        bd = L.bdev;
        xd = L.xdev;
    }
    Ctrl h = fresh_ctrl(o->maxit, o->tol);
    SSCG_CUDA(ctx, cudaMemcpyAsync(L.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * 3 + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    int rc = dispatch_pcg(ctx, mat, bd, xd, o->maxit, o->arith, L, &h, *prof, nullptr);
    if (rc) {
        delete prof;
        return rc;
    }
    if (o->flags & SSCG_HOST_VECTORS) {
        SSCG_CUDA(ctx, cudaMemcpyAsync(x, L.xdev, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    }
    if (h.status == SSCG_ERR_NONFINITE) {
        delete prof;
        return set_err(ctx, SSCG_ERR_NONFINITE, "non-finite right-hand side or x0");
    }
    if (h.status == SSCG_ERR_INVALID) {
        delete prof;
        return set_err(ctx, SSCG_ERR_INVALID, "right-hand side with max |b_i| outside [2^-30, 2^30], where double-float "
                                              "vectors and norms stay in FP32's exponent range; scale b or use f64");
    }
    if (info) fill_profile(info, *prof, h.step);
    delete prof;
    if (info) {
        info->status = h.status;
        info->outer_iters = h.step;
        info->equiv_iters = h.step;
        info->rel_res_recursive = h.relres;
        info->rel_res_true = h.zero_rhs ? 0.0 : sqrt(h.true_res2) / h.bnorm;
        int len = std::min(h.nhist, info->hist_cap);
        if (info->hist && len > 0)
            SSCG_CUDA(ctx, cudaMemcpy(info->hist, L.hist, len * sizeof(double), cudaMemcpyDeviceToHost));
        info->hist_len = info->hist ? len : 0;
    }
    return h.status;
}

int estimate_bounds(sscg_ctx* ctx, const sscg_mat* mat, int steps, const double* r0, void* ws, size_t ws_bytes,
                    double* lmin, double* lmax) {
    if (!mat || !lmin || !lmax || steps < 1 || steps > 100000)
        return set_err(ctx, SSCG_ERR_INVALID, "bad bounds-estimate arguments");
    size_t need = 0;
    bounds_workspace(mat, steps, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    PLayout L = pplan(mat, steps, 0, ws, ws_bytes);
    Carve c(ws, ws_bytes);
    c.used = L.bytes;
    double* bvec = c.take<double>(align_up((size_t)mat->n, 64));
    double* dwork = c.take<double>(2 * (size_t)steps + 2);
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n;
    if (r0) {
        SSCG_CUDA(ctx, cudaMemcpyAsync(bvec, r0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        k_splitmix_uniform<<<grid_for(ctx, n, 4), kThreads, 0, st>>>(n, 0x5EED5EEDull, bvec);
        SSCG_CUDA(ctx, cudaGetLastError());
    }
    Ctrl h = fresh_ctrl(steps, kLanczosTol);
    SSCG_CUDA(ctx, cudaMemcpyAsync(L.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    Prof prof(ctx, false);
    int rc = dispatch_pcg(ctx, mat, bvec, nullptr, steps, SSCG_ARITH_DF64, L, &h, prof, L.coef);
    if (rc) return rc;
    if (h.step < 1) return set_err(ctx, SSCG_BREAKDOWN, "Lanczos took no step");
    k_ritz<<<1, 32, 0, st>>>(L.coef, h.step, dwork, L.ctrl);
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(&h, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    *lmin = h.scratch[0];
    *lmax = h.scratch[1];
    return SSCG_OK;
}

int splitmix_uniform(sscg_ctx* ctx, int64_t n, uint64_t seed, double* out) {
    if (!out || n <= 0 || n >= INT32_MAX) return set_err(ctx, SSCG_ERR_INVALID, "bad length");
    k_splitmix_uniform<<<grid_for(ctx, n, 4), kThreads, 0, ctx->stream>>>((int)n, (unsigned long long)seed, out);
    SSCG_CUDA(ctx, cudaGetLastError());
    return SSCG_OK;
}

}  // namespace sscg
