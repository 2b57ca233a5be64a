// Mixed-precision s-step solve (Section IV, item (ii): higher precision for
// the moment-related computations).  The Krylov basis U that the
// matrix-powers kernel builds each outer step is stored in FP32 and
// multiplied with the FP32 matrix values; A U is formed from it with every
// product exact (products of two FP32 numbers) and the row sums in
// double-float, then stored in FP64.  The Gram sums are accumulated in FP64,
// the direction blocks P, AP (the method's memory across steps), x and r are
// FP64, and the s x s solves are FP64.  Every `replace_every` outer steps the
// residual is replaced by the true residual (Section IV, item (i)),
// r = r0 - A (x - x0) with r0 = b - A x0, computed in FP64 with the FP64
// matrix, and convergence is tested on it.  Blocks are formed by the
// direct-Gram path (any basis), because the moment recurrence of Algorithm 6
// assumes the exact recurrences that FP32 storage and residual replacement
// perturb.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "gram.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "small.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

// u = B^-1 r rounded to FP32 (B^-1 the array dinv, the constant dinv_c, or none).
__device__ __forceinline__ float mx_prec(const double* dinv, double dinv_c, int i, double r) {
    return (float)(dinv ? dinv[i] * r : (dinv_c != 0.0 ? dinv_c * r : r));
}

// r0 = r, u_1 = B^-1 r in FP32.
__global__ void k_mx_prep(int n, const double* __restrict__ r, double* __restrict__ r0,
                          const double* __restrict__ dinv, double dinv_c, float* __restrict__ u0, const Ctrl* ctrl) {
    if (__ldcg(&ctrl->done)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = r[i];
        r0[i] = v;
        u0[i] = mx_prec(dinv, dinv_c, i, v);
    }
}

// AU_j = A u_j from the FP32 u_j (exact products, double-float row sums),
// stored in FP64; u_{j+1} from B^-1 AU_j by the basis recurrence, rounded to
// FP32.  With DM != 0 the matrix's diagonal form (mode DM of spmv_dia_df;
// B^-1 the constant dinv_c or the identity, the FP32 basis columns carry
// margins).
template <int VM, int DM = 0>
__global__ void __launch_bounds__(kThreads, DM >= 2 ? 6 : 1)
    k_mx_level(MatView M, const float2* __restrict__ dinv_df, double dinv_c, const float* __restrict__ u_in,
               const float* __restrict__ u_prev, double* __restrict__ au_out, float* __restrict__ u_next, int j,
               Basis B, Ctrl* ctrl) {
    if (__ldcg(&ctrl->done)) return;
    if constexpr (DM != 0) {
        const df64 dcv = dinv_c != 0.0 ? df_from_double(dinv_c) : df_make(1.f, 0.f);
        const df64 cb = df_from_double(B.c);
        const df64 sc = df_from_double(B.cheb ? (j == 0 ? 1.0 : 2.0) / B.delta : 1.0);
        spmv_dia_df<DM>(M, u_in, [&](int i, df64 y0, df64 x0, df64 y1, df64 x1, bool has1) {
            if (has1) *reinterpret_cast<double2*>(au_out + i) = make_double2(df_to_double(y0), df_to_double(y1));
            else au_out[i] = df_to_double(y0);
            if (!u_next) return;
            df64 w0 = df_mul(dcv, y0), w1 = df_mul(dcv, y1);
            if (B.newton) {
                const df64 th = df_from_double(B.theta[j]), is = df_from_double(B.isig);
                w0 = df_mul(df_add(w0, df_neg(df_mul(th, x0))), is);
                w1 = df_mul(df_add(w1, df_neg(df_mul(th, x1))), is);
            } else if (B.cheb) {
                w0 = df_mul(df_add(w0, df_neg(df_mul(cb, x0))), sc);
                w1 = df_mul(df_add(w1, df_neg(df_mul(cb, x1))), sc);
                if (j > 0) {
                    df64 p0, p1;
                    DiaVec<float>::ld_pair(u_prev + i, p0, p1);
                    w0 = df_add(w0, df_neg(p0));
                    w1 = df_add(w1, df_neg(p1));
                }
            }
            if (has1) *reinterpret_cast<float2*>(u_next + i) = make_float2(w0.hi, w1.hi);
            else u_next[i] = w0.hi;
        });
        return;
    }
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    spmv_pipe<ArithDF64, VM, kStages>(
        M, smem, [&](int c) { return df_make(__ldg(u_in + c), 0.f); },
        [&](int row, df64 y) {
            au_out[row] = df_to_double(y);
            if (u_next) {
                df64 w = dinv_df ? df_mul(ArithDF64::ld(dinv_df + row), y) : y;
                df64 un = w;
                if (B.newton) {
                    un = df_mul(df_add(w, df_neg(df_mul(df_from_double(B.theta[j]), df_make(u_in[row], 0.f)))),
                                df_from_double(B.isig));
                } else if (B.cheb) {
                    df64 t = df_add(w, df_neg(df_mul(df_from_double(B.c), df_make(u_in[row], 0.f))));
                    un = j == 0 ? df_mul(t, df_from_double(1.0 / B.delta))
                                : df_add(df_mul(t, df_from_double(2.0 / B.delta)), df_make(-u_prev[row], 0.f));
                }
                u_next[row] = un.hi;
            }
        },
        ctrl);
}

// Closes an outer step in the last CTA: step count, history, stop test.
__device__ __forceinline__ void close_step(Ctrl* ctrl, double* hist, double rr) {
    int step = ctrl->step + 1;
    double rel = sqrt(rr) / ctrl->bnorm;
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

// P = U + P_old beta, AP = AU + AP_old beta, x += P alpha in FP64 (U FP32);
// with write_r also r -= AP alpha, u_1 = B^-1 r in FP32 and the stop test on
// the recursive residual (steps without residual replacement).  Without
// keep_ap (the residual replaced every step, and C formed from P_old and
// A U) A P is neither formed nor stored.
template <int SB>
__global__ void __launch_bounds__(kThreads) k_mx_update(int n, int ldn, int s, float* __restrict__ ublk,
                                                        const double* __restrict__ aublk,
                                                        double* __restrict__ p_new, const double* __restrict__ p_old,
                                                        double* __restrict__ xw, double* __restrict__ r,
                                                        const double* __restrict__ dinv, double dinv_c,
                                                        double* __restrict__ part, int first, int write_r, int keep_ap,
                                                        Ctrl* ctrl, double* __restrict__ hist) {
    if (__ldcg(&ctrl->done)) return;
    __shared__ double sb[SB * SB];
    __shared__ double sa[SB], sna[SB];
    __shared__ double red[kThreads / 32];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) sb[(e % s) + (e / s) * SB] = ctrl->beta[e];
    for (int e = threadIdx.x; e < s; e += blockDim.x) {
        sa[e] = ctrl->alpha[e];
        sna[e] = -ctrl->alpha[e];
    }
    __syncthreads();
    const size_t ld = (size_t)ldn;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // every load of the row is issued (L2 path) before its arithmetic
        double po[SB], apo[SB], uu[SB], au[SB];
#pragma unroll
        for (int l = 0; l < SB; l++)
            if (l < s) {
                uu[l] = (double)__ldcg(ublk + l * ld + i);
                if (keep_ap) au[l] = __ldcg(aublk + l * ld + i);
                if (!first) {
                    po[l] = __ldcg(p_old + l * ld + i);
                    if (keep_ap) apo[l] = __ldcg(p_old + (s + l) * ld + i);
                }
            }
        double xn = xw[i], rn = write_r ? r[i] : 0.0;
#pragma unroll
        for (int jj = 0; jj < SB; jj++) {
            if (jj < s) {
                double p = uu[jj];
                if (!first) {
#pragma unroll
                    for (int l = 0; l < SB; l++)
                        if (l < s) p = fma(po[l], sb[l + jj * SB], p);
                }
                __stcs(p_new + jj * ld + i, p);  // read again only next step
                xn = fma(p, sa[jj], xn);
                if (keep_ap) {
                    double ap = au[jj];
                    if (!first) {
#pragma unroll
                        for (int l = 0; l < SB; l++)
                            if (l < s) ap = fma(apo[l], sb[l + jj * SB], ap);
                    }
                    __stcs(p_new + (s + jj) * ld + i, ap);
                    if (write_r) rn = fma(ap, sna[jj], rn);
                }
            }
        }
        xw[i] = xn;
        if (write_r) {
            r[i] = rn;
            ublk[i] = mx_prec(dinv, dinv_c, i, rn);
            rr = fma(rn, rn, rr);
        }
    }
    if (!write_r) return;
    double v[1] = {rr};
    double out[1];
    block_sum<ArithF64, 1>(v, red, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
    if (!last_cta(&ctrl->ticket[2])) return;
    __shared__ double sh[32];
    double t = cta_sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) close_step(ctrl, hist, t);
}

// Residual replacement: r = r0 - A (x - x0) in FP64 with the FP64 matrix,
// u_1 = B^-1 r in FP32; the stop test on this true residual.  DM as in
// k_mx_level (x - x0 carries margins; B^-1 is then the constant dinv_c or the
// identity): 7 / 27 the FP64 Laplacian-class neighbour sum, 2 the clamped
// diagonal form, 0 CSR tiles.
template <int DM = 0>
__global__ void __launch_bounds__(kThreads) k_mx_replace(MatView M, const double* __restrict__ xw,
                                                         const double* __restrict__ r0, double* __restrict__ r,
                                                         const double* __restrict__ dinv, double dinv_c,
                                                         float* __restrict__ u0, double* __restrict__ part,
                                                         Ctrl* ctrl, double* __restrict__ hist) {
    if (__ldcg(&ctrl->done)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    __shared__ double red[kThreads / 32];
    double rr = 0.0;
    auto epi = [&](int row, double y) {
        const double rn = r0[row] - y;
        r[row] = rn;
        u0[row] = mx_prec(dinv, dinv_c, row, rn);
        rr = fma(rn, rn, rr);
    };
    bool ok = true;
    if constexpr (DM >= 7) {
        const double cc = M.dc[DM / 2], co = (double)M.dco;
        spmv_dia_lap_f64<DM>(M, xw, [&](int i, double S, double xc) { epi(i, fma(co, S, cc * xc)); });
    } else if constexpr (DM != 0) {
        spmv_dia<ArithF64>(M, [&](int c) { return __ldg(xw + c); }, epi);
    } else {
        ok = spmv_pipe<ArithF64, VAL_F64, kStages>(M, smem, [&](int c) { return __ldg(xw + c); }, epi, ctrl);
    }
    if (!ok) return;
    double v[1] = {rr};
    double out[1];
    block_sum<ArithF64, 1>(v, red, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
    if (!last_cta(&ctrl->ticket[3])) return;
    __shared__ double sh[32];
    double t = cta_sum_partials(part, gridDim.x, sh);
    if (threadIdx.x == 0) close_step(ctrl, hist, t);
}

struct MLayout {
    int64_t ldn;
    Ctrl* ctrl;
    double* hist;
    double* part;
    float* ublk;       // U, FP32, rebuilt every outer step
    double* aublk;     // A U, FP64
    double* pblk[2];   // P | AP, FP64, alternating new / old
    double* r;
    double* r0;
    double* xw;        // x - x0, FP64
    double* bdev;
    double* xdev;
    size_t bytes;
};

MLayout mplan(const sscg_mat* mat, const sscg_opts* o, void* base, size_t cap) {
    MLayout L{};
    L.ldn = (int64_t)align_up((size_t)mat->n, 64);
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)o->maxit + 2);
    L.part = c.take<double>((size_t)kMaxGrid * (o->s * (o->s + 1) / 2 + 2 * o->s + o->s * o->s + 4));
    // margins: the diagonal-form levels gather U and the replacement gathers
    // x - x0 without clamping
    const size_t g = dia_margin(mat);
    if (g) c.take<float>(g);
    L.ublk = c.take<float>((size_t)L.ldn * o->s);
    if (g) c.take<float>(g);
    L.aublk = c.take<double>((size_t)L.ldn * o->s);
    L.pblk[0] = c.take<double>((size_t)L.ldn * 2 * o->s);
    L.pblk[1] = c.take<double>((size_t)L.ldn * 2 * o->s);
    L.r = c.take<double>((size_t)L.ldn);
    L.r0 = c.take<double>((size_t)L.ldn);
    if (g) c.take<double>(g);
    L.xw = c.take<double>((size_t)L.ldn);
    if (g) c.take<double>(g);
    if (o->flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>((size_t)L.ldn);
        L.xdev = c.take<double>((size_t)L.ldn);
    }
    L.bytes = c.used;
    return L;
}

template <int VM, int SB, int DM>
int run_mixed(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o, const MLayout& L,
              Basis basis, Ctrl* hctrl, Prof& P) {
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n, s = o->s;
    const int cap = stage_cap(mat);
    const MatView M = mat_view(mat);
    const bool jac = mat->prec == SSCG_PREC_JACOBI;
    const float2* dinv_df = jac ? mat->dinv_df : nullptr;
    // B^-1 of the FP64 steps: the diagonal form's constant, or the array
    const double dinv_c = (DM != 0 && jac) ? mat->dia_dinv : 0.0;
    const double* dinv_d = (DM == 0 && jac) ? mat->dinv : nullptr;
    const size_t smem64 = stage_bytes<ArithF64, VAL_F64>(cap);
    const size_t smem_lvl = DM != 0 ? 0 : pipe_bytes<VAL_F32, kStages>(cap) + 128;  // the diagonal form stages nothing
    const size_t smem_rep = DM != 0 ? 0 : pipe_bytes<VAL_F64, kStages>(cap) + 128;
    const GramShape gs_full = gram_shape(s, 1, 1);
    const size_t smem_gram = std::max({2 * (size_t)gs_full.ncols * (kGramTile + 1) * sizeof(double), sizeof(SmallScratch),
                                       (size_t)kThreads * sizeof(double)});
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_init<ArithF64, VAL_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem64));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_mx_level<VAL_F32, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_lvl));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_gram<ArithF64, SB, float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_gram));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_mx_replace<DM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rep));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    const int Gi = occupancy_grid(ctx, k_init<ArithF64, VAL_F64>, smem64, n);
    const int Gl = occupancy_grid(ctx, k_mx_level<VAL_F32, DM>, smem_lvl, n);
    const int Gg = occupancy_grid(ctx, k_gram<ArithF64, SB, float>, smem_gram, n);
    const int Gu = occupancy_grid(ctx, k_mx_update<SB>, 0, n);
    const int Gr = occupancy_grid(ctx, k_mx_replace<DM>, smem_rep, n);
    const int Ge = occupancy_grid(ctx, k_mx_prep, 0, n);
    const int Gt = occupancy_grid(ctx, k_true_res, smem64, n);
    const size_t ld = (size_t)L.ldn;
    const int every = o->replace_every > 0 ? o->replace_every : 1;

    P.begin();
    k_init<ArithF64, VAL_F64><<<Gi, kThreads, smem64, st>>>(M, nullptr, b, x, L.xw, L.r, nullptr, L.part, L.ctrl,
                                                            L.hist);
    k_mx_prep<<<Ge, kThreads, 0, st>>>(n, L.r, L.r0, dinv_d, dinv_c, L.ublk, L.ctrl);
    P.end(FAM_INIT, 0);
    P.launches++;
    SSCG_CUDA(ctx, cudaGetLastError());
    const int per_chunk = std::max(1, 32 / (s + 3));
    ChunkPoll poll;
    SSCG_CUDA(ctx, poll.init());
    int launched = 0, err = 0;
    while (launched < o->maxit) {
        int c = std::min(per_chunk, o->maxit - launched);
        for (int q = 0; q < c; q++) {
            const int k = launched + q;
            float* ub = L.ublk;
            double* aub = L.aublk;
            double* pn = L.pblk[k & 1];
            double* po = L.pblk[(k + 1) & 1];
            P.begin();
            for (int j = 0; j < s; j++) {
                float* unext = j + 1 < s ? ub + (j + 1) * ld : nullptr;
                const float* uprev = j > 0 ? ub + (j - 1) * ld : nullptr;
                k_mx_level<VAL_F32, DM><<<Gl, kThreads, smem_lvl, st>>>(M, dinv_df, dinv_c, ub + j * ld, uprev,
                                                                        aub + j * ld, unext, j, basis, L.ctrl);
                if (j + 1 < s) P.launches++;
            }
            P.end(FAM_MPK, k);
            P.begin();
            // with the residual replaced every step, C = P_old^T (A U) and A P is never formed
            k_gram<ArithF64, SB, float><<<Gg, kThreads, smem_gram, st>>>(n, (int)L.ldn, s, nullptr, ub, aub, L.r,
                                                                         po, k > 0 ? 1 : 0, every == 1 ? 2 : 1,
                                                                         L.part, k, L.ctrl);
            P.end(FAM_DIR, k);
            const bool replace = (k + 1) % every == 0;
            P.begin();
            k_mx_update<SB><<<Gu, kThreads, 0, st>>>(n, (int)L.ldn, s, ub, aub, pn, po, L.xw, L.r, dinv_d, dinv_c,
                                                     L.part, k == 0, replace ? 0 : 1, every == 1 ? 0 : 1, L.ctrl,
                                                     L.hist);
            if (replace) {
                k_mx_replace<DM><<<Gr, kThreads, smem_rep, st>>>(M, L.xw, L.r0, L.r, dinv_d, dinv_c, ub, L.part,
                                                                 L.ctrl, L.hist);
                P.launches++;
            }
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
    k_export_x<ArithF64><<<Ge, kThreads, 0, st>>>(n, L.xw, x, L.ctrl);
    k_true_res<<<Gt, kThreads, smem64, st>>>(M, b, x, L.part, L.ctrl);
    P.end(FAM_FINAL, 0);
    P.launches++;
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(hctrl, L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return 0;
}

template <int VM, int DM>
int run_mixed_sb(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
                 const MLayout& L, Basis basis, Ctrl* hctrl, Prof& P) {
    if (o->s <= 4) return run_mixed<VM, 4, DM>(ctx, mat, b, x, o, L, basis, hctrl, P);
    if (o->s <= 8) return run_mixed<VM, 8, DM>(ctx, mat, b, x, o, L, basis, hctrl, P);
    return run_mixed<VM, 16, DM>(ctx, mat, b, x, o, L, basis, hctrl, P);
}

}  // namespace

int mixed_workspace(const sscg_mat* mat, const sscg_opts* o, size_t* bytes) {
    *bytes = mplan(mat, o, nullptr, 0).bytes;
    return 0;
}

int solve_mixed(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
                sscg_info* info, void* ws, size_t ws_bytes, double blo, double bhi) {
    size_t need = 0;
    mixed_workspace(mat, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, ws_bytes);
    MLayout L = mplan(mat, o, ws, ws_bytes);
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
    const int s = o->s;
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * 3 + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    int rc;
    // mplan() carves margins around U and x - x0 whenever the matrix has the diagonal form
    const int dm = dia_mode(mat, true);
    if (dm == 7) rc = run_mixed_sb<VAL_F32, 7>(ctx, mat, bd, xd, o, L, basis, &h, *prof);
    else if (dm == 27) rc = run_mixed_sb<VAL_F32, 27>(ctx, mat, bd, xd, o, L, basis, &h, *prof);
    else if (dm != 0) rc = run_mixed_sb<VAL_F32, 2>(ctx, mat, bd, xd, o, L, basis, &h, *prof);
    else if (mat->exact_fp32) rc = run_mixed_sb<VAL_F32, 0>(ctx, mat, bd, xd, o, L, basis, &h, *prof);
    else rc = run_mixed_sb<VAL_DF, 0>(ctx, mat, bd, xd, o, L, basis, &h, *prof);
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
