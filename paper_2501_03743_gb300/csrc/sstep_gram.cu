// The s-step method with Gram blocks formed directly (Section II-A:
// W_i = P_i^T A P_i, W_{i-1} beta_{i-1} + c_i = 0, W_i alpha_i = m_i), for
// any polynomial basis of the Krylov block and any preconditioner.  It is
// the path for the Chebyshev basis (Section IV names it as the stable
// alternative to the monomial basis) and for the Chebyshev polynomial
// preconditioner; the monomial basis with a diagonal preconditioner also
// runs here on request (SSCG_DIRECT_GRAM), as a cross-check of the moment
// recurrence.
//
// Per outer step:
//   s x k_level_gen : AU_j = A u_j; u_{j+1} from B^-1 AU_j by the basis
//                     recurrence (fused when B is diagonal, otherwise after
//                     the preconditioner kernels)
//   1 x k_gram      : G = U^T AU (lower triangle), m = U^T r,
//                     C = (A P_old)^T U, from a shared-memory tile of the
//                     block; the last CTA reduces them and solves
//                     W_old beta = -C, W = G + C^T beta, W alpha = m
//   1 x k_update    : the block updates of Algorithm 3
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "gram.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "prec.cuh"
#include "small.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

struct GLayout {
    int64_t ldn;
    Ctrl* ctrl;
    double* hist;
    double* part;
    void* blk[2];
    void* r;
    void* xw;
    void* w;
    void* tmp;
    double* bdev;
    double* xdev;
    size_t bytes;
};

GLayout gplan(const sscg_mat* mat, const sscg_opts* o, int G, void* base, size_t cap) {
    GLayout L{};
    L.ldn = (int64_t)align_up((size_t)mat->n, 64);
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)o->maxit + 2);
    GramShape gs = gram_shape(o->s, 1);
    L.part = c.take<double>((size_t)G * std::max(gs.E, 4));
    size_t blk = (size_t)L.ldn * 2 * o->s;
    // margins: the diagonal-form levels gather the U columns without clamping
    const size_t g = dia_margin(mat);
    if (g) c.take<double>(g);
    L.blk[0] = c.take<double>(blk);
    if (g) c.take<double>(g);
    L.blk[1] = c.take<double>(blk);
    if (g) c.take<double>(g);
    L.r = c.take<double>((size_t)L.ldn);
    L.xw = (o->arith == SSCG_ARITH_F64) ? nullptr : c.take<double>((size_t)L.ldn);
    L.w = c.take<double>((size_t)L.ldn);
    L.tmp = c.take<double>((size_t)L.ldn * 3);
    if (o->flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>((size_t)L.ldn);
        L.xdev = c.take<double>((size_t)L.ldn);
    }
    L.bytes = c.used;
    return L;
}

template <class A, int VM, int SB, int DM>
int run_gram(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o, const GLayout& L,
             const typename A::S* dinv, Basis basis, Ctrl* hctrl, Prof& P) {
    using S = typename A::S;
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n, s = o->s;
    const int cap = stage_cap(mat);
    const MatView M = mat_view(mat);
    const size_t smem = std::max(stage_bytes<A, VM>(cap), sizeof(SmallScratch));
    const size_t smem64 = stage_bytes<ArithF64, VAL_F64>(cap);
    const size_t smem_pipe = pipe_bytes<VM, kStages>(cap) + 128;
    const GramShape gs_full = gram_shape(s, 1);
    const size_t smem_gram = std::max({2 * (size_t)gs_full.ncols * (kGramTile + 1) * sizeof(S), sizeof(SmallScratch),
                                       (size_t)kThreads * sizeof(double)});
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_init<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const size_t smem_lv = DM != 0 ? 0 : smem_pipe;  // the diagonal form stages nothing
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_level_gen<A, VM, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_lv));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_cheb_step<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pipe));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_gram<A, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gram));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    const int Gi = occupancy_grid(ctx, k_init<A, VM>, smem, n);
    const int Gl = occupancy_grid(ctx, k_level_gen<A, VM, DM>, smem_lv, n);
    const int Gg = occupancy_grid(ctx, k_gram<A, SB>, smem_gram, n);
    size_t smem_upd = 0;
    int Gu = 0;
    if (int e = update_tma_setup<A, SB>(ctx, n, s, &smem_upd, &Gu)) return e;
    const int Ga = occupancy_grid(ctx, k_update_ap<A, SB>, 0, n);
    const int Ge = occupancy_grid(ctx, k_combine<A>, 0, n);
    const int Gt = occupancy_grid(ctx, k_true_res, smem64, n);
    const bool diag = mat->prec != SSCG_PREC_CHEB;
    ChebPrec<A, VM> cheb(diag ? 1 : mat->degree, diag ? 1.0 : mat->plmin, diag ? 2.0 : mat->plmax);
    const size_t ld = (size_t)L.ldn;
    S* blk[2] = {(S*)L.blk[0], (S*)L.blk[1]};
    S* r = (S*)L.r;
    S* xw = A::kind == 0 ? (S*)x : (S*)L.xw;
    S* w = (S*)L.w;
    S* tmp = (S*)L.tmp;
    const S* dvec = dinv;  // Jacobi scaling (null: B = I); the Chebyshev preconditioner scales by D^-1 too
    // under the diagonal form D is the constant diagonal value
    const double dinv_c = (DM != 0 && dinv) ? mat->dia_dinv : 0.0;

    P.begin();
    k_init<A, VM><<<Gi, kThreads, smem, st>>>(M, dvec, b, x, A::kind == 0 ? nullptr : xw, r, diag ? blk[0] : nullptr,
                                              L.part, L.ctrl, L.hist);
    if (!diag) P.launches += cheb.apply(M, dvec, r, blk[0], tmp, ld, Ge, Gl, smem_pipe, st, L.ctrl);
    P.end(FAM_INIT, 0);
    SSCG_CUDA(ctx, cudaGetLastError());

    const int per_chunk = std::max(1, 32 / (s + 2));
    ChunkPoll poll;
    SSCG_CUDA(ctx, poll.init());
    int launched = 0, err = 0;
    while (launched < o->maxit) {
        int c = std::min(per_chunk, o->maxit - launched);
        for (int q = 0; q < c; q++) {
            const int k = launched + q;
            S* bn = blk[k & 1];
            S* bo = blk[(k + 1) & 1];
            P.begin();
            for (int j = 0; j < s; j++) {
                S* unext = j + 1 < s ? bn + (j + 1) * ld : nullptr;
                const S* uprev = j > 0 ? bn + (j - 1) * ld : nullptr;
                k_level_gen<A, VM, DM><<<Gl, kThreads, smem_lv, st>>>(M, dvec, dinv_c, bn + j * ld, uprev,
                                                                       bn + (s + j) * ld, unext, j, basis,
                                                                       diag ? 1 : 0, L.ctrl);
                if (!diag && unext) {
                    P.launches += cheb.apply(M, dvec, bn + (s + j) * ld, w, tmp, ld, Ge, Gl, smem_pipe, st, L.ctrl);
                    k_combine<A><<<Ge, kThreads, 0, st>>>(n, w, bn + j * ld, uprev, unext, j, basis, L.ctrl);
                    P.launches++;
                }
                if (j + 1 < s) P.launches++;
            }
            P.end(FAM_MPK, k);
            P.begin();
            k_gram<A, SB><<<Gg, kThreads, smem_gram, st>>>(n, (int)L.ldn, s, bn, (const S*)nullptr, bn + s * ld, r,
                                                             bo, k > 0 ? 1 : 0, 0, L.part, k, L.ctrl);
            P.end(FAM_DIR, k);
            P.begin();
            if constexpr (SB <= 8)
                k_update_ap<A, SB><<<Ga, kThreads, 0, st>>>(n, (int)L.ldn, s, bn, bo, xw, r, dvec, L.part, k == 0,
                                                             diag ? 1 : 0, L.ctrl, L.hist);
            else
                k_update_tma<A, SB><<<Gu, kUpdRows, smem_upd, st>>>(n, (int)L.ldn, s, bn, bo, xw, r, dvec, L.part,
                                                                    k == 0, diag ? 1 : 0, L.ctrl, L.hist);
            if (!diag) P.launches += cheb.apply(M, dvec, r, bo, tmp, ld, Ge, Gl, smem_pipe, st, L.ctrl);
            P.end(FAM_UPDATE, k);
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
    if (A::kind != 0) k_export_x<A><<<Ge, kThreads, 0, st>>>(n, xw, x, L.ctrl);
    else k_zero_if_zero_rhs<<<Ge, kThreads, 0, st>>>(n, x, L.ctrl);
    k_true_res<<<Gt, kThreads, smem64, st>>>(M, b, x, L.part, L.ctrl);
    P.end(FAM_FINAL, 0);
    P.launches++;
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(hctrl, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return 0;
}

template <class A, int VM, int DM>
int run_gram_sb(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o, const GLayout& L,
                const typename A::S* dinv, Basis basis, Ctrl* hctrl, Prof& P) {
    if (o->s <= 4) return run_gram<A, VM, 4, DM>(ctx, mat, b, x, o, L, dinv, basis, hctrl, P);
    if (o->s <= 8) return run_gram<A, VM, 8, DM>(ctx, mat, b, x, o, L, dinv, basis, hctrl, P);
    return run_gram<A, VM, 16, DM>(ctx, mat, b, x, o, L, dinv, basis, hctrl, P);
}

}  // namespace

int gram_workspace(const sscg_mat* mat, const sscg_opts* o, size_t* bytes) {
    *bytes = gplan(mat, o, 8 * 160, nullptr, 0).bytes;
    return 0;
}

int solve_gram(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
               sscg_info* info, void* ws, size_t ws_bytes, double blo, double bhi) {
    size_t need = 0;
    gram_workspace(mat, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    GLayout L = gplan(mat, o, 8 * 160, ws, ws_bytes);
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
    h.s = o->s;
    h.tol = o->tol;
    SSCG_CUDA(ctx, cudaMemcpyAsync(L.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    const Basis basis = make_basis(o->basis, o->s, blo, bhi);
    if ((basis.cheb || basis.newton) && !(basis.delta > 0.0))
        return set_err(ctx, SSCG_ERR_INVALID, "empty basis interval");
    const int s = o->s;
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * 3 + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    const bool scale = mat->prec != SSCG_PREC_NONE;  // Jacobi and Chebyshev scale by D^-1
    int rc;
    if (o->arith == SSCG_ARITH_F64) {
        const double* d = scale ? mat->dinv : nullptr;
        if (s <= 4) rc = run_gram<ArithF64, VAL_F64, 4, 0>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
        else if (s <= 8) rc = run_gram<ArithF64, VAL_F64, 8, 0>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
        else rc = run_gram<ArithF64, VAL_F64, 16, 0>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
    } else {
        const float2* d = scale ? mat->dinv_df : nullptr;
        // the diagonal form serves the levels of a diagonal (or no) preconditioner; gplan()
        // carves margins around both blocks whenever the matrix has the form
        const int dm = mat->prec != SSCG_PREC_CHEB ? dia_mode(mat, true) : 0;
        if (dm == 7) rc = run_gram_sb<ArithDF64, VAL_F32, 7>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
        else if (dm == 27) rc = run_gram_sb<ArithDF64, VAL_F32, 27>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
        else if (dm != 0) rc = run_gram_sb<ArithDF64, VAL_F32, 2>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
        else if (mat->exact_fp32) rc = run_gram_sb<ArithDF64, VAL_F32, 0>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
        else rc = run_gram_sb<ArithDF64, VAL_DF, 0>(ctx, mat, bd, xd, o, L, d, basis, &h, *prof);
    }
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
        info->equiv_iters = (int64_t)h.step * s;
        info->rel_res_recursive = h.relres;
        info->rel_res_true = h.zero_rhs ? 0.0 : sqrt(h.true_res2) / h.bnorm;
        int len = std::min(h.nhist, info->hist_cap);
        if (info->hist && len > 0)
            SSCG_CUDA(ctx, cudaMemcpy(info->hist, L.hist, len * sizeof(double), cudaMemcpyDeviceToHost));
        info->hist_len = info->hist ? len : 0;
    }
    return h.status;
}

}  // namespace sscg

extern "C" int sscg_newton_shifts(int s, double lmin, double lmax, double* theta, double* sigma) {
    if (s < 1 || s > sscg::kMaxS || !(lmax > lmin) || !theta || !sigma) return SSCG_ERR_INVALID;
    const sscg::Basis b = sscg::make_basis(SSCG_BASIS_NEWTON, s, lmin, lmax);
    for (int j = 0; j + 1 < s; j++) theta[j] = b.theta[j];
    *sigma = 0.25 * (lmax - lmin);
    return SSCG_OK;
}
