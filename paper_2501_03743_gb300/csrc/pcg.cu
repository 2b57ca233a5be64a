// Preconditioned CG (Algorithm 1), the comparator of the s-step method, on
// the same SpMV tiles and arithmetic.  Per iteration:
//   k_pcg_spmv   : s_k = A p_k and p_k . s_k; last CTA forms alpha_k
//   k_pcg_update : x += alpha p, r -= alpha s, u = B^-1 r, r.r and u.r;
//                  last CTA forms beta_k and tests convergence
//   k_pcg_dir    : p_{k+1} = B^-1 r_{k+1} + beta_k p_k
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "spmv.cuh"

namespace sscg {

namespace {

__device__ __forceinline__ int done_of(const Ctrl* c) { return __ldcg(&c->done); }

template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_pcg_init(MatView M, const typename A::S* __restrict__ dinv,
                                                       const double* __restrict__ b, const double* __restrict__ x0,
                                                       typename A::S* __restrict__ xw, typename A::S* __restrict__ r,
                                                       typename A::S* __restrict__ p, double* __restrict__ part,
                                                       Ctrl* ctrl, double* __restrict__ hist) {
    using R = typename A::R;
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    __shared__ double red[3 * (kThreads / 32)];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    R bb = A::zero(), rr = A::zero(), ru = A::zero();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        R y;
        int row;
        bool live = tile_spmv<A, VM>(M, tile, [&](int c) { return A::from_d(__ldg(x0 + c)); }, y, row, smem, s_rp);
        if (live) {
            R bi = A::from_d(b[row]);
            R ri = A::sub(bi, y);
            R ui = dinv ? A::mul(A::ld(dinv + row), ri) : ri;
            if (xw) A::st(xw + row, A::zero());  // DF64 iterate holds x - x0
            A::st(r + row, ri);
            A::st(p + row, ui);
            bb = A::fma(bi, bi, bb);
            rr = A::fma(ri, ri, rr);
            ru = A::fma(ri, ui, ru);
        }
    }
    R v[3] = {bb, rr, ru};
    double out[3];
    block_sum<A, 3>(v, red, out);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = out[0];
        part[G + blockIdx.x] = out[1];
        part[2 * G + blockIdx.x] = out[2];
    }
    if (!last_cta(&ctrl->ticket[0])) return;
    __shared__ double sh[32];
    double sbb = cta_sum_partials(part, G, sh);
    double srr = cta_sum_partials(part + G, G, sh);
    double sru = cta_sum_partials(part + 2 * G, G, sh);
    if (threadIdx.x == 0) {
        ctrl->bnorm = sqrt(sbb);
        ctrl->rho = sru;
        ctrl->nhist = 1;
        if (sbb == 0.0) {
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

template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_pcg_spmv(MatView M, const typename A::S* __restrict__ p,
                                                       typename A::S* __restrict__ q, double* __restrict__ part,
                                                       Ctrl* ctrl) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    __shared__ double red[kThreads / 32];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    R pq = A::zero();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        R y;
        int row;
        bool live = tile_spmv<A, VM>(M, tile, [&](int c) { return A::ldg(p + c); }, y, row, smem, s_rp);
        if (live) {
            A::st(q + row, y);
            pq = A::fma(A::ldg(p + row), y, pq);
        }
    }
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
__global__ void __launch_bounds__(kThreads) k_pcg_update(int n, typename A::S* __restrict__ x,
                                                         typename A::S* __restrict__ r,
                                                         const typename A::S* __restrict__ p,
                                                         const typename A::S* __restrict__ q,
                                                         const typename A::S* __restrict__ dinv,
                                                         double* __restrict__ part, Ctrl* ctrl,
                                                         double* __restrict__ hist) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    __shared__ double red[2 * (kThreads / 32)];
    const R alpha = A::from_d(ctrl->pcg_alpha);
    R rr = A::zero(), ru = A::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R pi = A::ld(p + i);
        R xi = A::fma(alpha, pi, A::ld(x + i));
        R ri = A::sub(A::ld(r + i), A::mul(alpha, A::ld(q + i)));
        A::st(x + i, xi);
        A::st(r + i, ri);
        R ui = dinv ? A::mul(A::ld(dinv + i), ri) : ri;
        rr = A::fma(ri, ri, rr);
        ru = A::fma(ri, ui, ru);
    }
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
        ctrl->pcg_beta = sru / ctrl->rho;
        ctrl->rho = sru;
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

template <class A>
__global__ void __launch_bounds__(kThreads) k_pcg_dir(int n, typename A::S* __restrict__ p,
                                                      const typename A::S* __restrict__ r,
                                                      const typename A::S* __restrict__ dinv, const Ctrl* ctrl) {
    using R = typename A::R;
    if (done_of(ctrl)) return;
    const R beta = A::from_d(ctrl->pcg_beta);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R ri = A::ld(r + i);
        R ui = dinv ? A::mul(A::ld(dinv + i), ri) : ri;
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

struct PLayout {
    Ctrl* ctrl;
    double* hist;
    double* part;
    void *x, *r, *p, *q;
    double *bdev, *xdev;
    size_t bytes;
};

PLayout pplan(const sscg_mat* mat, const sscg_opts* o, int G, void* base, size_t cap) {
    PLayout L{};
    size_t ldn = align_up((size_t)mat->n, 64);
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)o->maxit + 2);
    L.part = c.take<double>((size_t)G * 4);
    L.x = c.take<double>(ldn);
    L.r = c.take<double>(ldn);
    L.p = c.take<double>(ldn);
    L.q = c.take<double>(ldn);
    if (o->flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>(ldn);
        L.xdev = c.take<double>(ldn);
    }
    L.bytes = c.used;
    return L;
}

int cap_of(const sscg_mat* m) {
    int cap = m->max_tile_nnz;
    if (cap > 8192) cap = 8192;
    if (cap < 32) cap = 32;
    return (cap + 31) / 32 * 32;
}

template <class A, int VM>
int run_pcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o, const PLayout& L,
            int G, const typename A::S* dinv, Ctrl* h, Prof& P) {
    using S = typename A::S;
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n;
    const int cap = cap_of(mat);
    MatView M;
    M.n = n;
    M.cap = cap;
    M.rowptr = mat->rowptr;
    M.col = mat->col;
    M.val = mat->val;
    M.vhi = mat->vhi;
    M.vlo = mat->vlo;
    const size_t smem = stage_bytes<A, VM>(cap), smem64 = stage_bytes<ArithF64, VAL_F64>(cap);
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pcg_init<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pcg_spmv<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_pcg_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    S* xw = A::kind == 0 ? (S*)x : (S*)L.x;
    S* r = (S*)L.r;
    S* p = (S*)L.p;
    S* q = (S*)L.q;
    P.begin();
    const int Gi = occupancy_grid(ctx, k_pcg_init<A, VM>, smem, n);
    const int Gs = occupancy_grid(ctx, k_pcg_spmv<A, VM>, smem, n);
    const int Gu = occupancy_grid(ctx, k_pcg_update<A>, 0, n);
    const int Gd = occupancy_grid(ctx, k_pcg_dir<A>, 0, n);
    const int Gt = occupancy_grid(ctx, k_pcg_true_res, smem64, n);
    k_pcg_init<A, VM><<<Gi, kThreads, smem, st>>>(M, dinv, b, x, A::kind == 0 ? nullptr : xw, r, p, L.part, L.ctrl,
                                                 L.hist);
    P.end(FAM_INIT, 0);
    SSCG_CUDA(ctx, cudaGetLastError());
    const int per_chunk = 16;
    cudaEvent_t ev[2];
    SSCG_CUDA(ctx, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    SSCG_CUDA(ctx, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    int launched = 0, chunk = 0, pending = -1, err = 0;
    while (launched < o->maxit) {
        int c = std::min(per_chunk, o->maxit - launched);
        for (int k = 0; k < c; k++) {
            const int it = launched + k;
            P.begin();
            k_pcg_spmv<A, VM><<<Gs, kThreads, smem, st>>>(M, p, q, L.part, L.ctrl);
            P.end(FAM_MPK, it);
            P.begin();
            k_pcg_update<A><<<Gu, kThreads, 0, st>>>(n, xw, r, p, q, dinv, L.part, L.ctrl, L.hist);
            P.end(FAM_UPDATE, it);
            P.begin();
            k_pcg_dir<A><<<Gd, kThreads, 0, st>>>(n, p, r, dinv, L.ctrl);
            P.end(FAM_DIR, it);
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
    k_pcg_export<A><<<G, kThreads, 0, st>>>(n, xw, x, L.ctrl);
    k_pcg_true_res<<<Gt, kThreads, smem64, st>>>(M, b, x, L.part, L.ctrl);
    P.end(FAM_FINAL, 0);
    P.launches++;
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(h, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return 0;
}

}  // namespace

int pcg_workspace(const sscg_mat* mat, const sscg_opts* o, size_t* bytes) {
    *bytes = pplan(mat, o, 8 * 160, nullptr, 0).bytes;
    return 0;
}

int solve_pcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
              sscg_info* info, void* ws, size_t ws_bytes) {
    if (!mat || !o || !b || !x) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    if (o->maxit < 0 || !(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad maxit or tol");
    if (o->arith != SSCG_ARITH_F64 && o->arith != SSCG_ARITH_DF64)
        return set_err(ctx, SSCG_ERR_INVALID, "arith %d not supported by PCG", o->arith);
    if (mat->prec != SSCG_PREC_NONE && mat->prec != SSCG_PREC_JACOBI)
        return set_err(ctx, SSCG_ERR_INVALID, "preconditioner %d not supported by this solver", mat->prec);
    size_t need = 0;
    pcg_workspace(mat, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    const int G = grid_for(ctx, mat->n, 8);
    PLayout L = pplan(mat, o, G, ws, ws_bytes);
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
    const bool jac = mat->prec == SSCG_PREC_JACOBI;
    int rc;
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * 3 + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    if (o->arith == SSCG_ARITH_F64)
        rc = run_pcg<ArithF64, VAL_F64>(ctx, mat, bd, xd, o, L, G, jac ? mat->dinv : nullptr, &h, *prof);
    else if (mat->exact_fp32)
        rc = run_pcg<ArithDF64, VAL_F32>(ctx, mat, bd, xd, o, L, G, jac ? mat->dinv_df : nullptr, &h, *prof);
    else
        rc = run_pcg<ArithDF64, VAL_DF>(ctx, mat, bd, xd, o, L, G, jac ? mat->dinv_df : nullptr, &h, *prof);
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

}  // namespace sscg
