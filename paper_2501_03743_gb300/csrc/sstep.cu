// Preconditioned s-step CG (Algorithm 3) on one GPU.
//
// Per outer step i the device runs
//   s x k_level  : one level of the preconditioned matrix-powers kernel
//                  (Algorithm 4): AU_j = A u_j and u_{j+1} = B^-1 A u_j, with
//                  the moments of Algorithm 5 accumulated in the epilogue as
//                  mu_{2j+1} = u_j . A u_j and mu_{2j+2} = (A u_j) . B^-1 (A u_j).
//                  The last level's last CTA reduces the moments and solves
//                  the s x s systems of Algorithm 6 on chip.
//   1 x k_update : the block updates of Algorithm 3 (P = U + P_old beta,
//                  AP = AU + AP_old beta, x += P alpha, r -= AP alpha) in one
//                  pass, fused with z = B^-1 r for the next step, ||r||^2 and
//                  mu_0 = r . z; its last CTA tests convergence.
// The two n x 2s blocks of Algorithm 3 (P1, P2) alternate between "new"
// and "old" with the step parity; P and AP overwrite U and AU in place.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "small.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

// One level of the matrix-powers kernel (Algorithm 4): y = A u_j, written to
// AU_j; u_{j+1} = B^-1 y (when u_next != null); moment partials
// mu_{2j+1} = u_j . y and mu_{2j+2} = y . B^-1 y.  With `last` set, the last
// CTA reduces mu_1..mu_{2s-1} and runs Algorithm 6.
template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_level(MatView M, const typename A::S* __restrict__ dinv,
                                                    const typename A::S* __restrict__ u_in,
                                                    typename A::S* __restrict__ au_out,
                                                    typename A::S* __restrict__ u_next, double* __restrict__ part,
                                                    int j, int s, int step, int last, Ctrl* ctrl) {
    using R = typename A::R;
    if (ctrl_done(ctrl)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    __shared__ double red[2 * (kThreads / 32)];
    R m1 = A::zero(), m2 = A::zero();
    const bool want_m2 = (2 * j + 2) <= (2 * s - 1);
    const bool ok = spmv_pipe<A, VM, kStages>(
        M, smem, [&](int c) { return A::ldg(u_in + c); },
        [&](int row, R y) {
            A::st(au_out + row, y);
            m1 = A::fma(A::ldg(u_in + row), y, m1);
            if (u_next || want_m2) {
                R z = dinv ? A::mul(A::ld(dinv + row), y) : y;
                if (u_next) A::st(u_next + row, z);
                m2 = A::fma(y, z, m2);
            }
        },
        ctrl);
    if (!ok) return;
    R v[2] = {m1, m2};
    double out[2];
    block_sum<A, 2>(v, red, out);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        part[(2 * j) * G + blockIdx.x] = out[0];
        part[(2 * j + 1) * G + blockIdx.x] = out[1];
    }
    if (!last) return;
    if (!last_cta(&ctrl->ticket[1])) return;
    cta_sum_rows(part, 2 * s - 1, G, [&](int e, double v) { ctrl->mu[e + 1] = v; });
    SmallScratch* sc = reinterpret_cast<SmallScratch*>(smem);  // staging buffer is free now
    if (threadIdx.x < 32) {
        int st = warp_sw_monomial(ctrl, s, step, sc);
        if (threadIdx.x == 0 && st != 0) {
            ctrl->status = st;
            ctrl->done = 1;
        }
    }
}

// ------------------------------------------------------------ host side

struct Layout {
    int64_t ldn;
    int G;
    Ctrl* ctrl;
    double* hist;
    double* part;
    void* blk[2];
    void* r;
    void* xw;
    double* bdev;
    double* xdev;
    size_t bytes;
};

int max_grid(const sscg_ctx* ctx) { return ctx->sm_count * 8; }

Layout plan(const sscg_mat* mat, const sscg_opts* o, int G, void* base, size_t cap) {
    Layout L{};
    L.ldn = (int64_t)align_up((size_t)mat->n, 64);
    L.G = G;
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)o->maxit + 2);
    L.part = c.take<double>((size_t)G * (2 * kMaxS + 4));
    size_t blk = (size_t)L.ldn * 2 * o->s;
    L.blk[0] = c.take<double>(blk);
    L.blk[1] = c.take<double>(blk);
    L.r = c.take<double>((size_t)L.ldn);
    L.xw = (o->arith == SSCG_ARITH_F64) ? nullptr : c.take<double>((size_t)L.ldn);
    if (o->flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>((size_t)L.ldn);
        L.xdev = c.take<double>((size_t)L.ldn);
    }
    L.bytes = c.used;
    return L;
}

MatView view_of(const sscg_mat* m, int cap) {
    MatView v;
    v.n = (int)m->n;
    v.cap = cap;
    v.rowptr = m->rowptr;
    v.col = m->col;
    v.val = m->val;
    v.vhi = m->vhi;
    v.vlo = m->vlo;
    return v;
}


template <class A, int VM, int SB>
int run_sstep(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
              const Layout& L, const typename A::S* dinv, Ctrl* hctrl, Prof& P) {
    using S = typename A::S;
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n, s = o->s, G = L.G;
    const int cap = stage_cap(mat);
    MatView M = view_of(mat, cap);
    const size_t smem = std::max(stage_bytes<A, VM>(cap), sizeof(SmallScratch));
    const size_t smem_pipe = std::max(pipe_bytes<VM, kStages>(cap), sizeof(SmallScratch)) + 128;
    const size_t smem64 = stage_bytes<ArithF64, VAL_F64>(cap);
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_init<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_level<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_pipe));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    S* blk[2] = {(S*)L.blk[0], (S*)L.blk[1]};
    S* r = (S*)L.r;
    S* xw = A::kind == 0 ? (S*)x : (S*)L.xw;
    const size_t ld = (size_t)L.ldn;

    P.begin();
    const int Gi = occupancy_grid(ctx, k_init<A, VM>, smem, n);
    const int Gl = occupancy_grid(ctx, k_level<A, VM>, smem_pipe, n);
    size_t smem_upd = 0;
    int Gu = 0;
    if (int e = update_tma_setup<A, SB>(ctx, n, s, &smem_upd, &Gu)) return e;
    const int Gt = occupancy_grid(ctx, k_true_res, smem64, n);
    k_init<A, VM><<<Gi, kThreads, smem, st>>>(M, dinv, b, x, A::kind == 0 ? nullptr : xw, r, blk[0], L.part,
                                              L.ctrl, L.hist);
    P.end(FAM_INIT, 0);
    SSCG_CUDA(ctx, cudaGetLastError());

    const int per_chunk = std::max(1, 32 / (s + 1));
    cudaEvent_t ev[2];
    SSCG_CUDA(ctx, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    SSCG_CUDA(ctx, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    int launched = 0, chunk = 0, pending = -1;
    int err = 0;
    while (launched < o->maxit) {
        int c = std::min(per_chunk, o->maxit - launched);
        for (int q = 0; q < c; q++) {
            const int k = launched + q;
            S* bn = blk[k & 1];
            S* bo = blk[(k + 1) & 1];
            for (int j = 0; j < s; j++) {
                P.begin();
                k_level<A, VM><<<Gl, kThreads, smem_pipe, st>>>(M, dinv, bn + j * ld, bn + (s + j) * ld,
                                                          j + 1 < s ? bn + (j + 1) * ld : nullptr, L.part, j, s, k,
                                                          j == s - 1, L.ctrl);
                P.end(FAM_MPK, k);
            }
            P.begin();
            k_update_tma<A, SB><<<Gu, kUpdRows, smem_upd, st>>>(n, (int)L.ldn, s, bn, bo, xw, r, dinv, L.part,
                                                                k == 0, 1, L.ctrl, L.hist);
            P.end(FAM_UPDATE, k);
        }
        if (cudaGetLastError() != cudaSuccess) { err = 1; break; }
        launched += c;
        const int slot = chunk & 1;
        SSCG_CUDA(ctx, cudaMemcpyAsync((void*)(ctx->pinned + slot), &L.ctrl->done, sizeof(int),
                                       cudaMemcpyDeviceToHost, st));
        SSCG_CUDA(ctx, cudaEventRecord(ev[slot], st));
        if (pending >= 0) {
            SSCG_CUDA(ctx, cudaEventSynchronize(ev[pending & 1]));
            if (ctx->pinned[pending & 1]) break;
        }
        pending = chunk++;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (err) return set_err(ctx, SSCG_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    P.begin();
    if (A::kind != 0) k_export_x<A><<<G, kThreads, 0, st>>>(n, xw, x, L.ctrl);
    else k_zero_if_zero_rhs<<<G, kThreads, 0, st>>>(n, x, L.ctrl);
    k_true_res<<<Gt, kThreads, smem64, st>>>(M, b, x, L.part, L.ctrl);
    P.end(FAM_FINAL, 0);
    P.launches++;
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(hctrl, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return 0;
}

}  // namespace

int sstep_workspace(const sscg_mat* mat, const sscg_opts* o, size_t* bytes) {
    // The grid is at most 8 CTAs per SM of any GB300-class part; size for 8 * 160.
    Layout L = plan(mat, o, 8 * 160, nullptr, 0);
    *bytes = L.bytes;
    return 0;
}

static int check_opts(sscg_ctx* ctx, const sscg_mat* mat, const sscg_opts* o) {
    if (!mat || !o) return set_err(ctx, SSCG_ERR_INVALID, "null matrix or options");
    if (o->s < 1 || o->s > kMaxS) return set_err(ctx, SSCG_ERR_INVALID, "s = %d outside 1..%d", o->s, kMaxS);
    if (o->maxit < 0) return set_err(ctx, SSCG_ERR_INVALID, "maxit < 0");
    if (!(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "tol must be >= 0");
    if (o->arith != SSCG_ARITH_F64 && o->arith != SSCG_ARITH_DF64)
        return set_err(ctx, SSCG_ERR_INVALID, "arith %d not supported by this solver", o->arith);
    if (o->basis != SSCG_BASIS_MONOMIAL)
        return set_err(ctx, SSCG_ERR_INVALID, "the moment recurrence needs the monomial basis");
    if (mat->prec != SSCG_PREC_NONE && mat->prec != SSCG_PREC_JACOBI)
        return set_err(ctx, SSCG_ERR_INVALID, "preconditioner %d not supported by this solver", mat->prec);
    return 0;
}

int solve_sstep(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
                sscg_info* info, void* ws, size_t ws_bytes) {
    int e = check_opts(ctx, mat, o);
    if (e) return e;
    if (!b || !x) return set_err(ctx, SSCG_ERR_INVALID, "null b or x");
    size_t need = 0;
    sstep_workspace(mat, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    const int G = grid_for(ctx, mat->n, 8);
    Layout L = plan(mat, o, G, ws, ws_bytes);
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
    const bool jac = mat->prec == SSCG_PREC_JACOBI;
    int rc;
    const int s = o->s;
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * (s + 1) + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    if (o->arith == SSCG_ARITH_F64) {
        const double* dinv = jac ? mat->dinv : nullptr;
        if (s <= 4) rc = run_sstep<ArithF64, VAL_F64, 4>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
        else if (s <= 8) rc = run_sstep<ArithF64, VAL_F64, 8>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
        else rc = run_sstep<ArithF64, VAL_F64, 16>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
    } else {
        const float2* dinv = jac ? mat->dinv_df : nullptr;
        if (mat->exact_fp32) {
            if (s <= 4) rc = run_sstep<ArithDF64, VAL_F32, 4>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
            else if (s <= 8) rc = run_sstep<ArithDF64, VAL_F32, 8>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
            else rc = run_sstep<ArithDF64, VAL_F32, 16>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
        } else {
            if (s <= 4) rc = run_sstep<ArithDF64, VAL_DF, 4>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
            else if (s <= 8) rc = run_sstep<ArithDF64, VAL_DF, 8>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
            else rc = run_sstep<ArithDF64, VAL_DF, 16>(ctx, mat, bd, xd, o, L, dinv, &h, *prof);
        }
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
