// Kernels shared by the two s-step drivers (moment recurrence of
// Algorithm 6, and directly formed Gram blocks): the initial residual, the
// block updates of Algorithm 3, the export of x and the true residual.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "spmv.cuh"

namespace sscg {

namespace {

__device__ __forceinline__ int ctrl_done(const Ctrl* c) { return __ldcg(&c->done); }

// r = b - A x0 (x0 and b FP64), x_w = x0, z = B^-1 r -> u0; ||b||^2 and
// max |b_i| (in FP64 whatever the arithmetic), ||r||^2, mu_0 = r . z; the
// last CTA initialises the control block.  A double-float solve whose
// right-hand side lies outside [kDfRhsMin, kDfRhsMax] stops with
// SSCG_ERR_INVALID before its first step.  `part` holds 4 G doubles.
template <class A, int VM>
__global__ void __launch_bounds__(kThreads) k_init(MatView M, const typename A::S* __restrict__ dinv,
                                                   const double* __restrict__ b, const double* __restrict__ x0,
                                                   typename A::S* __restrict__ xw, typename A::S* __restrict__ r,
                                                   typename A::S* __restrict__ u0, double* __restrict__ part,
                                                   Ctrl* ctrl, double* __restrict__ hist) {
    using R = typename A::R;
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    __shared__ double red[3 * (kThreads / 32)];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    R rr = A::zero(), rz = A::zero();
    double bb = 0.0, bmax = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        R y;
        int row;
        bool live = tile_spmv<A, VM>(M, tile, [&](int c) { return A::from_d(__ldg(x0 + c)); }, y, row, smem, s_rp);
        if (live) {
            const double bd = b[row];
            R bi = A::from_d(bd);
            R ri = A::sub(bi, y);
            if (xw) A::st(xw + row, A::zero());  // DF64 iterate holds x - x0
            A::st(r + row, ri);
            bb = fma(bd, bd, bb);
            bmax = fmax(bmax, fabs(bd));
            rr = A::fma(ri, ri, rr);
            if (u0) {  // null: the preconditioner is applied by separate kernels
                R zi = dinv ? A::mul(A::ld(dinv + row), ri) : ri;
                A::st(u0 + row, zi);
                rz = A::fma(ri, zi, rz);
            }
        }
    }
    R v[2] = {rr, rz};
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
    double srz = cta_sum_partials(part + 2 * G, G, sh);
    const double smax = cta_max_partials(part + 3 * G, G, sh);
    if (threadIdx.x == 0) {
        ctrl->bnorm = sqrt(sbb);
        ctrl->mu[0] = srz;
        if (A::kind != 0 && isfinite(sbb) && sbb != 0.0 && (smax < kDfRhsMin || smax > kDfRhsMax)) {
            ctrl->status = SSCG_ERR_INVALID;
            ctrl->done = 1;
        } else if (sbb == 0.0) {
            ctrl->zero_rhs = 1;
            ctrl->relres = 0.0;
            hist[0] = 0.0;
            ctrl->nhist = 1;
            ctrl->status = 0;
            ctrl->done = 1;
        } else {
            double rel = sqrt(srr) / ctrl->bnorm;
            ctrl->relres = rel;
            hist[0] = rel;
            ctrl->nhist = 1;
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

// Block updates of Algorithm 3 (P = U + P_old beta, AP = AU + AP_old beta,
// x += P alpha, r -= AP alpha, z = B^-1 r and ||r||^2, mu_0 = r . z for the
// next step) fed by bulk copies: a CTA of kUpdRows threads
// takes tiles of kUpdRows rows; thread 0 copies each tile's slice of every
// input column (U, AU, P_old, AP_old, r and 1/diag) into one of two shared
// memory stages with cp.async.bulk, completing on the stage's mbarrier, so
// the bytes in flight do not depend on the registers a thread holds.  x is
// read with ordinary loads (it may be the caller's exact-length vector).
constexpr int kUpdRows = 128;

template <int SB>
__host__ __device__ constexpr int upd_cols(int s) {
    return 4 * s + 2;  // U, AU, P_old, AP_old, r, 1/diag
}

template <class A, int SB>
__host__ __device__ constexpr size_t upd_smem(int s) {
    return 16 + 2 * (size_t)upd_cols<SB>(s) * kUpdRows * sizeof(typename A::S);
}

template <class A, int SB>
__global__ void __launch_bounds__(kUpdRows) k_update_tma(int n, int ldn, int s, typename A::S* __restrict__ blk_new,
                                                          typename A::S* __restrict__ blk_old,
                                                          typename A::S* __restrict__ x, typename A::S* __restrict__ r,
                                                          const typename A::S* __restrict__ dinv,
                                                          double* __restrict__ part, int first, int write_z,
                                                          Ctrl* ctrl, double* __restrict__ hist) {
    using R = typename A::R;
    using S = typename A::S;
    if (ctrl_done(ctrl)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    S* stage0 = reinterpret_cast<S*>(smem + 16);
    const int ncols = upd_cols<SB>(s);
    const size_t stage_elems = (size_t)ncols * kUpdRows;
    __shared__ R sb[SB * SB];
    __shared__ R sa[SB];
    __shared__ double red[2 * (kThreads / 32)];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) sb[(e % s) + (e / s) * SB] = A::from_d(ctrl->beta[e]);
    for (int e = threadIdx.x; e < s; e += blockDim.x) sa[e] = A::from_d(ctrl->alpha[e]);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const size_t ld = (size_t)ldn;
    const int ntiles = (n + kUpdRows - 1) / kUpdRows;
    const int G = gridDim.x;
    const int my = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + G - 1) / G : 0;
    // column c of the stage: 0..s-1 U, s..2s-1 AU, 2s..3s-1 P_old, 3s..4s-1 AP_old, 4s r, 4s+1 1/diag
    auto src = [&](int c) -> const S* {
        if (c < 2 * s) return blk_new + c * ld;
        if (c < 4 * s) return blk_old + (c - 2 * s) * ld;
        return c == 4 * s ? r : dinv;
    };
    auto issue = [&](int k) {
        const int r0 = ((int)blockIdx.x + k * G) * kUpdRows, rows = min(kUpdRows, n - r0);
        const unsigned bytes = (unsigned)(((rows + 1) & ~1) * sizeof(S));  // 16-byte multiple
        S* st = stage0 + (size_t)(k & 1) * stage_elems;
        unsigned tx = 0;
        for (int c = 0; c < ncols; c++) {
            const bool need = (c < 2 * s) || (c < 4 * s && !first) || c == 4 * s || (c == 4 * s + 1 && dinv);
            if (need) tx += bytes;
        }
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[k & 1], tx);
        for (int c = 0; c < ncols; c++) {
            const bool need = (c < 2 * s) || (c < 4 * s && !first) || c == 4 * s || (c == 4 * s + 1 && dinv);
            if (need) bulk_g2s(st + (size_t)c * kUpdRows, src(c) + r0, bytes, &bar[k & 1]);
        }
    };
    if (threadIdx.x == 0 && my > 0) issue(0);
    R rr = A::zero(), rz = A::zero();
    for (int k = 0; k < my; k++) {
        if (threadIdx.x == 0 && k + 1 < my) issue(k + 1);
        const bool ok = __syncthreads_and(mbar_wait(&bar[k & 1], (unsigned)(k >> 1) & 1u));
        if (!ok) {
            if (threadIdx.x == 0) {
                ctrl->status = 3;  // SSCG_TIMEOUT
                __threadfence();
                atomicExch(&ctrl->done, 1);
                if (k + 1 < my) mbar_wait(&bar[(k + 1) & 1], (unsigned)((k + 1) >> 1) & 1u);
            }
            __syncthreads();
            return;
        }
        const S* st = stage0 + (size_t)(k & 1) * stage_elems;
        const int r0 = ((int)blockIdx.x + k * G) * kUpdRows, rows = min(kUpdRows, n - r0);
        const int t = threadIdx.x;
        if (t < rows) {
            const int i = r0 + t;
            R xa = A::zero(), ra = A::zero();
#pragma unroll
            for (int jj = 0; jj < SB; jj++) {
                if (jj < s) {
                    R p = A::ld(st + (size_t)jj * kUpdRows + t);
                    R ap = A::ld(st + (size_t)(s + jj) * kUpdRows + t);
                    if (!first) {
#pragma unroll
                        for (int l = 0; l < SB; l++)
                            if (l < s) {
                                const R b = sb[l + jj * SB];
                                p = A::fma(A::ld(st + (size_t)(2 * s + l) * kUpdRows + t), b, p);
                                ap = A::fma(A::ld(st + (size_t)(3 * s + l) * kUpdRows + t), b, ap);
                            }
                    }
                    A::st(blk_new + jj * ld + i, p);
                    A::st(blk_new + (s + jj) * ld + i, ap);
                    xa = A::fma(p, sa[jj], xa);
                    ra = A::fma(ap, sa[jj], ra);
                }
            }
            R xn = A::add(A::ld(x + i), xa);
            R rn = A::sub(A::ld(st + (size_t)(4 * s) * kUpdRows + t), ra);
            A::st(x + i, xn);
            A::st(r + i, rn);
            rr = A::fma(rn, rn, rr);
            if (write_z) {
                R z = dinv ? A::mul(A::ld(st + (size_t)(4 * s + 1) * kUpdRows + t), rn) : rn;
                A::st(blk_old + i, z);
                rz = A::fma(rn, z, rz);
            }
        }
        __syncthreads();  // stage k & 1 may be refilled
    }
    R v[2] = {rr, rz};
    double out[2];
    block_sum<A, 2>(v, red, out);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = out[0];
        part[G + blockIdx.x] = out[1];
    }
    if (!last_cta(&ctrl->ticket[2])) return;
    __shared__ double sh[32];
    double srr = cta_sum_partials(part, G, sh);
    double srz = cta_sum_partials(part + G, G, sh);
    if (threadIdx.x == 0) {
        int step = ctrl->step + 1;
        double rel = sqrt(srr) / ctrl->bnorm;
        ctrl->step = step;
        ctrl->relres = rel;
        ctrl->mu[0] = srz;
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

// The same update (U, AU, P_old, AP_old, r, 1/diag in; P, AP, x, r and z out)
// with each thread taking whole rows (grid-stride) and issuing every load of
// a row through L2 before its arithmetic; P and AP are written with streaming
// stores (read again only in the next step).  Used by the direct-Gram path
// for s <= 8 (the row's 4s values stay in registers).
template <class A, int SB>
__global__ void __launch_bounds__(kThreads, 2) k_update_ap(int n, int ldn, int s, typename A::S* __restrict__ blk_new,
                                                        typename A::S* __restrict__ blk_old,
                                                        typename A::S* __restrict__ x, typename A::S* __restrict__ r,
                                                        const typename A::S* __restrict__ dinv,
                                                        double* __restrict__ part, int first, int write_z,
                                                        Ctrl* ctrl, double* __restrict__ hist) {
    using R = typename A::R;
    using S = typename A::S;
    if (ctrl_done(ctrl)) return;
    __shared__ R sb[SB * SB];
    __shared__ R sa[SB];
    __shared__ double red[2 * (kThreads / 32)];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) sb[(e % s) + (e / s) * SB] = A::from_d(ctrl->beta[e]);
    for (int e = threadIdx.x; e < s; e += blockDim.x) sa[e] = A::from_d(ctrl->alpha[e]);
    __syncthreads();
    const size_t ld = (size_t)ldn;
    R rr = A::zero(), rz = A::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R u[SB], au[SB], po[SB], apo[SB];
#pragma unroll
        for (int l = 0; l < SB; l++)
            if (l < s) {
                u[l] = A::ldcg(blk_new + l * ld + i);
                au[l] = A::ldcg(blk_new + (s + l) * ld + i);
                if (!first) {
                    po[l] = A::ldcg(blk_old + l * ld + i);
                    apo[l] = A::ldcg(blk_old + (s + l) * ld + i);
                }
            }
        const R r0 = A::ldcg(r + i), x0 = A::ldcg(x + i);
        const R dv = dinv ? A::ldcg(dinv + i) : A::zero();
        R xa = A::zero(), ra = A::zero();
#pragma unroll
        for (int jj = 0; jj < SB; jj++) {
            if (jj < s) {
                R p = u[jj], ap = au[jj];
                if (!first) {
#pragma unroll
                    for (int l = 0; l < SB; l++)
                        if (l < s) {
                            const R b = sb[l + jj * SB];
                            p = A::fma(po[l], b, p);
                            ap = A::fma(apo[l], b, ap);
                        }
                }
                A::st_stream(blk_new + jj * ld + i, p);
                A::st_stream(blk_new + (s + jj) * ld + i, ap);
                xa = A::fma(p, sa[jj], xa);
                ra = A::fma(ap, sa[jj], ra);
            }
        }
        const R xn = A::add(x0, xa);
        const R rn = A::sub(r0, ra);
        A::st(x + i, xn);
        A::st(r + i, rn);
        rr = A::fma(rn, rn, rr);
        if (write_z) {
            const R z = dinv ? A::mul(dv, rn) : rn;
            A::st(blk_old + i, z);  // U_1 of the next step (P_old_1 of this row is already read)
            rz = A::fma(rn, z, rz);
        }
    }
    R v[2] = {rr, rz};
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
    double srz = cta_sum_partials(part + G, G, sh);
    if (threadIdx.x == 0) {
        int step = ctrl->step + 1;
        double rel = sqrt(srr) / ctrl->bnorm;
        ctrl->step = step;
        ctrl->relres = rel;
        ctrl->mu[0] = srz;
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

// Launch geometry of k_update_tma: dynamic shared memory and a persistent
// grid from the occupancy of its 128-thread CTAs.
template <class A, int SB>
inline int update_tma_setup(sscg_ctx* ctx, int64_t n, int s, size_t* smem, int* grid) {
    *smem = upd_smem<A, SB>(s) + 128;
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_update_tma<A, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
    int per_sm = 0;
    SSCG_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_tma<A, SB>, kUpdRows, *smem));
    int64_t g = (int64_t)ctx->sm_count * (per_sm < 1 ? 1 : per_sm);
    int64_t tiles = (n + kUpdRows - 1) / kUpdRows;
    if (g > tiles) g = tiles;
    if (g > kMaxGrid) g = kMaxGrid;
    *grid = g < 1 ? 1 : (int)g;
    return 0;
}

// End of the z / Q block updates: the grid's sums of ||r||^2 and mu_0 = r . z
// (rr and rz of this thread; without a diagonal array rz holds sum z^2 and r =
// diag_c z), the step count, the residual history and the stopping test.
template <class A>
__device__ __forceinline__ void update_q_finish(typename A::R rr, typename A::R rz, bool has_diag, double diag_c,
                                                double* red, double* __restrict__ part, Ctrl* ctrl,
                                                double* __restrict__ hist) {
    if (!has_diag) {  // r = d z: ||r||^2 = d^2 sum z^2, mu_0 = d sum z^2 (d = 1 without a preconditioner)
        const typename A::R dcst = A::from_d(diag_c);
        if (diag_c != 0.0) rz = A::mul(dcst, rz);
        rr = diag_c != 0.0 ? A::mul(dcst, rz) : rz;
    }
    typename A::R v[2] = {rr, rz};
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
    double srz = cta_sum_partials(part + G, G, sh);
    if (threadIdx.x == 0) {
        int step = ctrl->step + 1;
        double rel = sqrt(srr) / ctrl->bnorm;
        ctrl->step = step;
        ctrl->relres = rel;
        ctrl->mu[0] = srz;
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

// Block update carrying z = D^-1 r and Q = D^-1 A P (diagonal
// preconditioner D, or none).  With u_{j+1} = D^-1 A u_j the level kernel
// never stores A U: D^-1 A U_{1..s} = U_{2..s+1}, so
//   P_j = U_j + sum_l P_old_l beta_lj,   Q_j = U_{j+1} + sum_l Q_old_l beta_lj,
//   x += P alpha,   z -= Q alpha   (r -= A P alpha multiplied by D^-1),
// the same recurrences as Algorithm 3 written for D^-1 r and D^-1 A P.
// ||r||^2 = sum (d z)^2 and mu_0 = r . z = sum d z^2 for the next step
// (d the array diag, or the constant diag_c when diag is null, or 1).
// Block layout (2s+1 columns): 0..s U_1..U_{s+1}, s+1..2s Q; after the
// update columns 0..s-1 hold P.  z for the next step goes to column 0 of
// the old block (whose P_old_1 the stage already holds).
// Each thread takes whole rows (grid-stride) and issues all of a row's 3s+2
// loads (through L2, ld.global.cg) before its arithmetic: measured on the
// GB300 at 256^3, s = 4, this moves the (5s+4) vectors at 6.5 TB/s, where
// staging 128-row column slices by bulk copy into two shared-memory stages
// reached 4.6 TB/s.  P and Q are written with streaming stores (they are
// read again only in the next step, from HBM).
template <class A, int SB>
__global__ void __launch_bounds__(kThreads) k_update_q(int n, int ldn, int s, typename A::S* __restrict__ blk_new,
                                                       typename A::S* __restrict__ blk_old,
                                                       typename A::S* __restrict__ x,
                                                       const typename A::S* __restrict__ diag, double diag_c,
                                                       double* __restrict__ part, int first, Ctrl* ctrl,
                                                       double* __restrict__ hist) {
    using R = typename A::R;
    using S = typename A::S;
    if (ctrl_done(ctrl)) return;
    __shared__ R sb[SB * SB];
    __shared__ R sa[SB];
    __shared__ double red[2 * (kThreads / 32)];
    __shared__ R sna[SB];
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) sb[(e % s) + (e / s) * SB] = A::from_d(ctrl->beta[e]);
    for (int e = threadIdx.x; e < s; e += blockDim.x) {
        sa[e] = A::from_d(ctrl->alpha[e]);
        sna[e] = A::from_d(-ctrl->alpha[e]);
    }
    __syncthreads();
    const size_t ld = (size_t)ldn;
    R rr = A::zero(), rz = A::zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        R u[SB + 1], po[SB], qo[SB];
#pragma unroll
        for (int c = 0; c <= SB; c++)
            if (c <= s) u[c] = A::ldcg(blk_new + c * ld + i);
        if (!first) {
#pragma unroll
            for (int l = 0; l < SB; l++)
                if (l < s) {
                    po[l] = A::ldcg(blk_old + l * ld + i);
                    qo[l] = A::ldcg(blk_old + (s + 1 + l) * ld + i);
                }
        }
        // x and z accumulate onto their old values: x += P alpha, z += Q (-alpha)
        R xn = A::ldcg(x + i), zn = u[0];
#pragma unroll
        for (int jj = 0; jj < SB; jj++) {
            if (jj < s) {
                R p = u[jj];
                R q = u[jj + 1];
                if (!first) {
#pragma unroll
                    for (int l = 0; l < SB; l++)
                        if (l < s) {
                            const R b = sb[l + jj * SB];
                            p = A::fma(po[l], b, p);
                            q = A::fma(qo[l], b, q);
                        }
                    A::st_stream(blk_new + jj * ld + i, p);
                }
                A::st_stream(blk_new + (s + 1 + jj) * ld + i, q);
                xn = A::fma(p, sa[jj], xn);
                zn = A::fma(q, sna[jj], zn);
            }
        }
        A::st(x + i, xn);
        A::st(blk_old + i, zn);  // U_1 of the next step (P_old_1 already read)
        if (diag) {
            const R rn = A::mul(A::ldcg(diag + i), zn);
            rr = A::fma(rn, rn, rr);
            rz = A::fma(rn, zn, rz);
        } else {
            rz = A::fma(zn, zn, rz);  // sum z^2; scaled by the constant diagonal below
        }
    }
    update_q_finish<A>(rr, rz, diag != nullptr, diag_c, red, part, ctrl, hist);
}

// Per-thread asynchronous copies of 8 bytes global -> shared (cp.async),
// completion tracked per thread by commit groups.
__device__ __forceinline__ void row_cp8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void row_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void row_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void row_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int S>
__host__ __device__ constexpr size_t fix_row_smem() {
    return 2 * (size_t)(3 * S + 2) * kThreads * sizeof(double);
}

// The FP64 block update of k_update_q with P and Q formed as fixed-point dot
// products on the integer multipliers (fixsum.cuh), for block sizes S <= 6:
//   P_j = U_j + sum_l P_old_l beta_lj,   Q_j = U_{j+1} + sum_l Q_old_l beta_lj
// take 3 (S + 1) 32 x 32 -> 64-bit multiply-adds each in place of S FP64 FMAs
// (a GB300 retires about 53 of those per SM and clock against 2 FP64
// operations).  A row's values U_1..U_{S+1}, P_old and Q_old share one
// alignment exponent; each column j of the coefficients [1; beta_0j ..
// beta_{S-1}j] has its own.  x += P alpha and z -= Q alpha stay FP64 FMAs on
// the rounded P and Q, as in k_update_q.  A row holding a NaN, an infinity or
// only values below 2^-961, or whose entries could leave the normal range,
// takes the FP64 FMAs of k_update_q; so does every row when a coefficient is
// not finite.  Not for the first step (no P_old, Q_old).
template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_update_fix(int n, int ldn, double* __restrict__ blk_new,
                                                            double* __restrict__ blk_old, double* __restrict__ x,
                                                            const double* __restrict__ diag, double diag_c,
                                                            double* __restrict__ part, Ctrl* ctrl,
                                                            double* __restrict__ hist) {
    static_assert(S + 1 <= kFixMaxTerms, "the 64-bit sums of fixsum.cuh hold at most kFixMaxTerms products");
    if (ctrl_done(ctrl)) return;
    __shared__ double sb[S * S];
    __shared__ double sa[S];
    __shared__ double sna[S];
    __shared__ FixLimbs scf[S][S + 1];
    __shared__ int sfc[S];
    __shared__ double red[2 * (kThreads / 32)];
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) sb[e] = ctrl->beta[e];
    for (int e = threadIdx.x; e < S; e += blockDim.x) {
        sa[e] = ctrl->alpha[e];
        sna[e] = -ctrl->alpha[e];
    }
    __syncthreads();
    if (threadIdx.x < S) sfc[threadIdx.x] = fix_coef_column<S>(sb, threadIdx.x, scf[threadIdx.x]);
    __syncthreads();
    int fc[S];
#pragma unroll
    for (int j = 0; j < S; j++) fc[j] = sfc[j];
    int Elo, Ehi;  // the rows that take the fixed point
    fix_row_range<S>(fc, &Elo, &Ehi);
    const size_t ld = (size_t)ldn;
    double rr = 0.0, rz = 0.0;
    // each thread copies its next row's 3S+2 values (U_1..U_{S+1}, P_old, Q_old,
    // x) into its own slots of one of two shared-memory buffers while it
    // computes the current row
    extern __shared__ __align__(16) double rowbuf[];
    constexpr int NCOL = 3 * S + 2;
    const int stride = gridDim.x * blockDim.x;
    auto issue = [&](int i, int b) {
        double* d = rowbuf + (size_t)b * NCOL * kThreads + threadIdx.x;
#pragma unroll
        for (int c = 0; c <= S; c++) row_cp8(d + c * kThreads, blk_new + c * ld + i);
#pragma unroll
        for (int l = 0; l < S; l++) {
            row_cp8(d + (S + 1 + l) * kThreads, blk_old + l * ld + i);
            row_cp8(d + (2 * S + 1 + l) * kThreads, blk_old + (S + 1 + l) * ld + i);
        }
        row_cp8(d + (3 * S + 1) * kThreads, x + i);
        row_commit();
    };
    int k = 0;
    if (blockIdx.x * blockDim.x + threadIdx.x < n) issue(blockIdx.x * blockDim.x + threadIdx.x, 0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride, k++) {
        if ((unsigned)i + (unsigned)stride < (unsigned)n) {  // no overflow: i, stride < 2^31
            issue(i + stride, (k + 1) & 1);
            row_wait_prior();
        } else {
            row_wait_all();
        }
        double u[S + 1], po[S], qo[S];
        const double* d = rowbuf + (size_t)(k & 1) * NCOL * kThreads + threadIdx.x;
#pragma unroll
        for (int c = 0; c <= S; c++) u[c] = d[c * kThreads];
#pragma unroll
        for (int l = 0; l < S; l++) {
            po[l] = d[(S + 1 + l) * kThreads];
            qo[l] = d[(2 * S + 1 + l) * kThreads];
        }
        double xn = d[(3 * S + 1) * kThreads];
        double zn = u[0];
        // the row exponent E: the largest exponent field of its values (sign
        // cleared, as an integer), shared by the P and Q columns
        double p[S], q[S];
        unsigned hmax = 0;
#pragma unroll
        for (int c = 0; c <= S; c++) hmax = max(hmax, (unsigned)__double2hiint(u[c]) & 0x7FF00000u);
#pragma unroll
        for (int l = 0; l < S; l++)
            hmax = max(hmax, max((unsigned)__double2hiint(po[l]) & 0x7FF00000u,
                                 (unsigned)__double2hiint(qo[l]) & 0x7FF00000u));
        const int E = (int)(hmax >> 20);
        if (E >= Elo && E <= Ehi) {
            FixLimbs au[S + 1], ap[S], aq[S];
#pragma unroll
            for (int c = 0; c <= S; c++) au[c] = fix_align((uint64_t)__double_as_longlong(u[c]), E);
#pragma unroll
            for (int l = 0; l < S; l++) {
                ap[l] = fix_align((uint64_t)__double_as_longlong(po[l]), E);
                aq[l] = fix_align((uint64_t)__double_as_longlong(qo[l]), E);
            }
#pragma unroll
            for (int j = 0; j < S; j++) {
                FixAcc a1, a2;
                fix_mad(a1, au[j], scf[j][0]);
                fix_mad(a2, au[j + 1], scf[j][0]);
#pragma unroll
                for (int l = 0; l < S; l++) {
                    fix_mad(a1, ap[l], scf[j][1 + l]);
                    fix_mad(a2, aq[l], scf[j][1 + l]);
                }
                p[j] = fix_pack_cvt(fix_total(a1), fix_dot_e0(E, fc[j]));
                q[j] = fix_pack_cvt(fix_total(a2), fix_dot_e0(E, fc[j]));
            }
        } else {  // FP64 FMAs, as k_update_q
            double v[S];
#pragma unroll
            for (int j = 0; j < S; j++) v[j] = u[j];
            fma_update_group<S>(v, po, sb, p);
#pragma unroll
            for (int j = 0; j < S; j++) v[j] = u[j + 1];
            fma_update_group<S>(v, qo, sb, q);
        }
#pragma unroll
        for (int j = 0; j < S; j++) {
            __stcs(blk_new + j * ld + i, p[j]);
            xn = ::fma(p[j], sa[j], xn);
            __stcs(blk_new + (S + 1 + j) * ld + i, q[j]);
            zn = ::fma(q[j], sna[j], zn);
        }
        x[i] = xn;
        blk_old[i] = zn;  // U_1 of the next step (P_old_1 already read)
        if (diag) {
            const double rn = __ldcg(diag + i) * zn;
            rr = ::fma(rn, rn, rr);
            rz = ::fma(rn, zn, rz);
        } else {
            rz = ::fma(zn, zn, rz);
        }
    }
    update_q_finish<ArithF64>(rr, rz, diag != nullptr, diag_c, red, part, ctrl, hist);
}

template <class A, int SB>
inline int update_q_setup(sscg_ctx* ctx, int64_t n, int s, size_t* smem, int* grid) {
    (void)s;
    *smem = 0;
    *grid = occupancy_grid(ctx, k_update_q<A, SB>, 0, n);
    return 0;
}

// x = x0 + (x - x0): the DF64 iterate carries the correction to x0, so x0
// keeps every bit when no step is taken; 0 when b = 0.
template <class A>
__global__ void k_export_x(int n, const typename A::S* __restrict__ xw, double* __restrict__ x, const Ctrl* ctrl) {
    const int zero = ctrl->zero_rhs;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = zero ? 0.0 : x[i] + A::to_d(A::ld(xw + i));
}

// F64 iterates in place: only b = 0 needs x cleared.
__global__ void k_zero_if_zero_rhs(int n, double* __restrict__ x, const Ctrl* ctrl) {
    if (!ctrl->zero_rhs) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

// ||b - A x||^2 in FP64 (the true residual reported at exit).
__global__ void __launch_bounds__(kThreads) k_true_res(MatView M, const double* __restrict__ b,
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


}  // namespace

}  // namespace sscg
