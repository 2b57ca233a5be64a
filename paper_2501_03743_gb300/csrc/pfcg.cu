// PFCG-NN (Algorithm 2): Notay's flexible preconditioned CG with one global
// reduction per iteration, the comparison solver of the paper.  Per
// iteration k the device runs
//   k_pfcg_dots   : w_k = A u_k (u_k = B^-1 r_k, stored by the previous
//                   update) and the coupled dot products alpha_k = u.r,
//                   beta_k = u.w, gamma_k = u.s_{k-1}, plus ||r_k||^2; its
//                   last CTA tests ||r_k|| / ||b|| < tol (the test Algorithm 2
//                   makes after its update, taken here before the next
//                   update, so the iterate returned is the same x_k) and forms
//                   rho_k = beta_k - gamma_k^2 / rho_{k-1}, the coefficients
//                   gamma_k / rho_{k-1} and alpha_k / rho_k
//   k_pfcg_update : the coupled axpys p = u - (gamma/rho_{k-1}) p,
//                   s = w - (gamma/rho_{k-1}) s, x += (alpha/rho_k) p,
//                   r -= (alpha/rho_k) s, and u_{k+1} = B^-1 r_{k+1}
// Algorithm 2's first step is the same iteration with p_{-1} = s_{-1} = 0
// (gamma_0 = 0, rho_0 = beta_0, p_0 = u_0, s_0 = w_0).
// B is the Jacobi preconditioner or the identity; the matrix is multiplied in
// CSR tiles or its diagonal form (in FP64, the Laplacian-class neighbour sum).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

// r = b - A x0, u = B^-1 r, p = s = 0; ||b||^2, max |b_i| in FP64.
template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_pfcg_init(MatView M, const typename A::S* __restrict__ dinv,
                                                        double dinv_c, const double* __restrict__ b,
                                                        const double* __restrict__ x0, typename A::S* __restrict__ xw,
                                                        typename A::S* __restrict__ r, typename A::S* __restrict__ u,
                                                        typename A::S* __restrict__ p, typename A::S* __restrict__ s,
                                                        double* __restrict__ part, Ctrl* ctrl,
                                                        double* __restrict__ hist) {
    using R = typename A::R;
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    __shared__ double red[kThreads / 32];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    const R dc = A::from_d(dinv_c);
    double bb = 0.0, bmax = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        R y;
        int row;
        const bool live =
            tile_spmv<A, VM>(M, tile, [&](int c) { return A::from_d(__ldg(x0 + c)); }, y, row, smem, s_rp);
        if (live) {
            const double bd = b[row];
            const R ri = A::sub(A::from_d(bd), y);
            A::st(r + row, ri);
            A::st(u + row, dinv ? A::mul(A::ld(dinv + row), ri) : (dinv_c != 0.0 ? A::mul(dc, ri) : ri));
            A::st(p + row, A::zero());
            A::st(s + row, A::zero());
            if (xw) A::st(xw + row, A::zero());  // double-float iterate holds x - x0
            bb = fma(bd, bd, bb);
            bmax = fmax(bmax, fabs(bd));
        }
    }
    double vb[1] = {bb}, ob[1];
    block_sum<ArithF64, 1>(vb, red, ob);
    const double bm = block_max(isfinite(bmax) ? bmax : 0.0, red);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ob[0];
        part[G + blockIdx.x] = bm;
    }
    if (!last_cta(&ctrl->ticket[0])) return;
    __shared__ double sh[32];
    const double sbb = cta_sum_partials(part, G, sh);
    const double smax = cta_max_partials(part + G, G, sh);
    if (threadIdx.x == 0) {
        ctrl->bnorm = sqrt(sbb);
        ctrl->rho = 1.0;  // rho_{-1}: any nonzero value (gamma_0 = 0)
        if (!isfinite(sbb)) {
            ctrl->status = SSCG_ERR_NONFINITE;
            ctrl->done = 1;
        } else if (A::kind != 0 && sbb != 0.0 && (smax < kDfRhsMin || smax > kDfRhsMax)) {
            ctrl->status = SSCG_ERR_INVALID;
            ctrl->done = 1;
        } else if (sbb == 0.0) {
            ctrl->zero_rhs = 1;
            ctrl->status = 0;
            ctrl->done = 1;
            hist[0] = 0.0;
            ctrl->nhist = 1;
        }
    }
}

// w = A u and the coupled dot products (see the file comment).
template <class A, int VM, int DM>
__global__ void __launch_bounds__(kThreads, dia_min_blocks<A, DM>())
    k_pfcg_dots(MatView M, const typename A::S* __restrict__ u, const typename A::S* __restrict__ r,
                const typename A::S* __restrict__ s, typename A::S* __restrict__ w, double* __restrict__ part,
                Ctrl* ctrl, double* __restrict__ hist) {
    using R = typename A::R;
    if (ctrl_done(ctrl)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    __shared__ double red[4 * (kThreads / 32)];
    R al = A::zero(), be = A::zero(), ga = A::zero(), rr = A::zero();
    auto epi = [&](int i, R y, R ui) {
        A::st(w + i, y);
        const R ri = A::ld(r + i);
        al = A::fma(ui, ri, al);
        be = A::fma(ui, y, be);
        ga = A::fma(ui, A::ld(s + i), ga);
        rr = A::fma(ri, ri, rr);
    };
    bool ok = true;
    if constexpr (DM >= 7 && A::kind == 0) {
        const double cc = M.dc[DM / 2], co = (double)M.dco;
        if (co == -1.0)
            spmv_dia_lap_f64<DM>(M, u, [&](int i, double S, double uc) { epi(i, fma(cc, uc, -S), uc); });
        else
            spmv_dia_lap_f64<DM>(M, u, [&](int i, double S, double uc) { epi(i, fma(co, S, cc * uc), uc); });
    } else if constexpr (DM != 0) {
        spmv_dia<A>(M, [&](int c) { return A::ldg(u + c); }, [&](int i, R y) { epi(i, y, A::ld(u + i)); });
    } else {
        ok = spmv_pipe<A, VM, kStages>(
            M, smem, [&](int c) { return A::ldg(u + c); }, [&](int i, R y) { epi(i, y, A::ld(u + i)); }, ctrl);
    }
    if (!ok) return;
    R v[4] = {al, be, ga, rr};
    double out[4];
    block_sum<A, 4>(v, red, out);
    const int G = gridDim.x;
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; q++) part[q * G + blockIdx.x] = out[q];
    if (!last_cta(&ctrl->ticket[1])) return;
    __shared__ double sh[32];
    const double a = cta_sum_partials(part, G, sh);
    const double bt = cta_sum_partials(part + G, G, sh);
    const double g = cta_sum_partials(part + 2 * G, G, sh);
    const double r2 = cta_sum_partials(part + 3 * G, G, sh);
    if (threadIdx.x == 0) {
        const int step = ctrl->step;
        const double rel = sqrt(r2) / ctrl->bnorm;
        ctrl->relres = rel;
        hist[step] = rel;
        ctrl->nhist = step + 1;
        const double rho = ctrl->rho;
        const double rho_new = bt - g * g / rho;
        if (!isfinite(rel)) {
            ctrl->status = step == 0 ? SSCG_ERR_NONFINITE : 2;
            ctrl->done = 1;
        } else if (rel < ctrl->tol) {
            ctrl->status = 0;
            ctrl->done = 1;
        } else if (step >= ctrl->maxit) {
            ctrl->status = 1;
            ctrl->done = 1;
        } else if (!(rho_new > 0.0) || !isfinite(rho_new) || !isfinite(a)) {
            ctrl->status = 2;  // SSCG_BREAKDOWN: B or A not positive definite on the Krylov space
            ctrl->done = 1;
        } else {
            ctrl->pcg_beta = g / rho;       // gamma_k / rho_{k-1}
            ctrl->pcg_alpha = a / rho_new;  // alpha_k / rho_k
            ctrl->rho = rho_new;
            ctrl->step = step + 1;
        }
    }
}

// The coupled axpys and u = B^-1 r of the new residual.
template <class A>
__global__ void __launch_bounds__(kThreads) k_pfcg_update(int n, typename A::S* __restrict__ p,
                                                          typename A::S* __restrict__ s,
                                                          const typename A::S* __restrict__ w,
                                                          typename A::S* __restrict__ x, typename A::S* __restrict__ r,
                                                          typename A::S* __restrict__ u,
                                                          const typename A::S* __restrict__ dinv, double dinv_c,
                                                          const Ctrl* ctrl) {
    using R = typename A::R;
    if (ctrl_done(ctrl)) return;
    const R nc = A::from_d(-ctrl->pcg_beta), a = A::from_d(ctrl->pcg_alpha), na = A::from_d(-ctrl->pcg_alpha);
    const R dc = A::from_d(dinv_c);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const R pi = A::fma(nc, A::ld(p + i), A::ld(u + i));
        const R si = A::fma(nc, A::ld(s + i), A::ld(w + i));
        A::st(p + i, pi);
        A::st(s + i, si);
        A::st(x + i, A::fma(a, pi, A::ld(x + i)));
        const R ri = A::fma(na, si, A::ld(r + i));
        A::st(r + i, ri);
        A::st(u + i, dinv ? A::mul(A::ld(dinv + i), ri) : (dinv_c != 0.0 ? A::mul(dc, ri) : ri));
    }
}

struct FLayout {
    Ctrl* ctrl;
    double* hist;
    double* part;
    void *x, *r, *u, *p, *s, *w;
    double *bdev, *xdev;
    size_t bytes;
};

FLayout fplan(const sscg_mat* mat, int maxit, unsigned flags, void* base, size_t cap) {
    FLayout L{};
    const size_t ldn = align_up((size_t)mat->n, 64);
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)maxit + 2);
    L.part = c.take<double>((size_t)kMaxGrid * 4);
    L.x = c.take<double>(ldn);
    L.r = c.take<double>(ldn);
    // margins around u: the diagonal-form SpMV gathers it without clamping
    const size_t g = dia_margin(mat);
    if (g) c.take<double>(g);
    L.u = c.take<double>(ldn);
    if (g) c.take<double>(g);
    L.p = c.take<double>(ldn);
    L.s = c.take<double>(ldn);
    L.w = c.take<double>(ldn);
    if (flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>(ldn);
        L.xdev = c.take<double>(ldn);
    }
    L.bytes = c.used;
    return L;
}

template <class A, int VM, int DM>
int run_pfcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, int maxit, const FLayout& L,
             const typename A::S* dinv, Ctrl* h, Prof& P) {
    using S = typename A::S;
    constexpr bool DIA = DM != 0;
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n;
    const MatView M = mat_view(mat);
    const size_t smem = stage_bytes<A, VM>(M.cap), smem64 = stage_bytes<ArithF64, VAL_F64>(M.cap);
    const size_t smem_d = DIA ? 128 : pipe_bytes<VM, kStages>(M.cap) + 128;
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pfcg_init<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pfcg_dots<A, VM, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_d));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    const int Gi = occupancy_grid(ctx, k_pfcg_init<A, VM>, smem, n);
    const int Gd = occupancy_grid(ctx, k_pfcg_dots<A, VM, DM>, smem_d, n);
    const int Gu = occupancy_grid(ctx, k_pfcg_update<A>, 0, n);
    const int Gt = occupancy_grid(ctx, k_true_res, smem64, n);
    // with the diagonal form, a Jacobi D is the constant diagonal value
    const bool cd = DIA && dinv != nullptr;
    const S* dinv_it = cd ? nullptr : dinv;
    const double dinv_c = cd ? mat->dia_dinv : 0.0;
    S* xw = (A::kind == 0) ? (S*)x : (S*)L.x;
    S* r = (S*)L.r;
    S* u = (S*)L.u;
    S* p = (S*)L.p;
    S* s = (S*)L.s;
    S* w = (S*)L.w;
    P.begin();
    k_pfcg_init<A, VM><<<Gi, kThreads, smem, st>>>(M, dinv_it, dinv_c, b, x, A::kind == 0 ? nullptr : xw, r, u, p, s,
                                                   L.part, L.ctrl, L.hist);
    P.end(FAM_INIT, 0);
    SSCG_CUDA(ctx, cudaGetLastError());
    const int per_chunk = 16;
    ChunkPoll poll;
    SSCG_CUDA(ctx, poll.init());
    int launched = 0, err = 0;
    // maxit iterations need maxit + 1 dots launches (the last one only tests)
    while (launched <= maxit) {
        const int c = std::min(per_chunk, maxit + 1 - launched);
        for (int k = 0; k < c; k++) {
            const int it = launched + k;
            P.begin();
            k_pfcg_dots<A, VM, DM><<<Gd, kThreads, smem_d, st>>>(M, u, r, s, w, L.part, L.ctrl, L.hist);
            P.end(FAM_MPK, it);
            if (it < maxit) {
                P.begin();
                k_pfcg_update<A><<<Gu, kThreads, 0, st>>>(n, p, s, w, xw, r, u, dinv_it, dinv_c, L.ctrl);
                P.end(FAM_UPDATE, it);
            }
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
    P.begin();
    if (A::kind != 0) k_export_x<A><<<Gu, kThreads, 0, st>>>(n, xw, x, L.ctrl);
    else k_zero_if_zero_rhs<<<Gu, kThreads, 0, st>>>(n, x, L.ctrl);
    k_true_res<<<Gt, kThreads, smem64, st>>>(M, b, x, L.part, L.ctrl);
    P.end(FAM_FINAL, 0);
    P.launches++;
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(h, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return 0;
}

int dispatch_pfcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, int maxit, int arith,
                  const FLayout& L, Ctrl* h, Prof& P) {
    const bool jac = mat->prec == SSCG_PREC_JACOBI;
    const bool dia = mat->dia != 0;
    if (arith == SSCG_ARITH_F64) {
        const double* d = jac ? mat->dinv : nullptr;
        // the layout carves margins around u, the only vector the SpMV gathers
        const int dm = dia ? dia_mode(mat, true) : 0;
        if (dm == 7) return run_pfcg<ArithF64, VAL_F64, 7>(ctx, mat, b, x, maxit, L, d, h, P);
        if (dm == 27) return run_pfcg<ArithF64, VAL_F64, 27>(ctx, mat, b, x, maxit, L, d, h, P);
        if (dm != 0) return run_pfcg<ArithF64, VAL_F64, 1>(ctx, mat, b, x, maxit, L, d, h, P);
        return run_pfcg<ArithF64, VAL_F64, 0>(ctx, mat, b, x, maxit, L, d, h, P);
    }
    const float2* d = jac ? mat->dinv_df : nullptr;
    if (dia) return run_pfcg<ArithDF64, VAL_F32, 1>(ctx, mat, b, x, maxit, L, d, h, P);
    if (mat->exact_fp32) return run_pfcg<ArithDF64, VAL_F32, 0>(ctx, mat, b, x, maxit, L, d, h, P);
    return run_pfcg<ArithDF64, VAL_DF, 0>(ctx, mat, b, x, maxit, L, d, h, P);
}

}  // namespace

}  // namespace sscg

using namespace sscg;

extern "C" int sscg_pfcg_workspace_bytes(const sscg_mat* m, const sscg_opts* o, size_t* bytes) {
    if (!m || !o || !bytes || o->maxit < 0) return SSCG_ERR_INVALID;
    *bytes = fplan(m, o->maxit, o->flags, nullptr, 0).bytes;
    return SSCG_OK;
}

extern "C" int sscg_pfcg_solve(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
                               sscg_info* info, void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (!mat || !o || !b || !x) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    if (o->maxit < 0 || !(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad maxit or tol");
    if (o->arith != SSCG_ARITH_F64 && o->arith != SSCG_ARITH_DF64)
        return set_err(ctx, SSCG_ERR_INVALID, "arith %d not supported by PFCG", o->arith);
    if (o->arith != SSCG_ARITH_F64 && mat->out_of_f32)
        return set_err(ctx, SSCG_ERR_INVALID, "matrix values lie outside FP32's normal range, which double-float "
                                              "arithmetic carries; use f64");
    if (mat->prec != SSCG_PREC_NONE && mat->prec != SSCG_PREC_JACOBI)
        return set_err(ctx, SSCG_ERR_INVALID, "PFCG takes the Jacobi preconditioner or none");
    size_t need = 0;
    sscg_pfcg_workspace_bytes(mat, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    FLayout L = fplan(mat, o->maxit, o->flags, ws, ws_bytes);
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
    Ctrl h;
    memset(&h, 0, sizeof(h));
    h.status = 1;
    h.maxit = o->maxit;
    h.s = 1;
    h.tol = o->tol;
    SSCG_CUDA(ctx, cudaMemcpyAsync(L.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * 2 + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    const int rc = dispatch_pfcg(ctx, mat, bd, xd, o->maxit, o->arith, L, &h, *prof);
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
        const int len = std::min(h.nhist, info->hist_cap);
        if (info->hist && len > 0)
            SSCG_CUDA(ctx, cudaMemcpy(info->hist, L.hist, len * sizeof(double), cudaMemcpyDeviceToHost));
        info->hist_len = info->hist ? len : 0;
    }
    return h.status;
}
