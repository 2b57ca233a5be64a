// Preconditioned s-step CG (Algorithm 3) on one GPU, monomial basis, B
// diagonal (Jacobi) or the identity.
//
// The device carries z = B^-1 r and Q = B^-1 A P instead of r and A P (the
// recurrences of Algorithm 3 multiplied by B^-1), so the matrix-powers
// levels never store A U: B^-1 A U_{1..s} = U_{2..s+1}.  Per outer step i:
//   s x k_level    : one level of the preconditioned matrix-powers kernel
//                    (Algorithm 4): u_{j+1} = B^-1 A u_j, with the moments of
//                    Algorithm 5 accumulated in the epilogue as
//                    mu_{2j+1} = u_j . A u_j and mu_{2j+2} = (A u_j) . B^-1 (A u_j).
//                    The last level's last CTA reduces the moments and solves
//                    the s x s systems of Algorithm 6 on chip.
//   1 x k_update_q : the block updates P = U + P_old beta, Q = U_{2..s+1} +
//                    Q_old beta, x += P alpha, z -= Q alpha in one pass, with
//                    ||r||^2 and mu_0 = r . z of the new residual; its last CTA
//                    tests convergence.  In FP64 at s <= 6 every step after the
//                    first runs k_update_fix instead: the same update with P
//                    and Q formed as fixed-point dot products on the integer
//                    multipliers (fixsum.cuh).
// A block holds 2s+1 columns (U_1..U_{s+1} | Q); the two blocks (the P1, P2 of
// Algorithm 3) alternate between "new" and "old" with the step parity.  With
// SSCG_FUSED_MPK the levels run in the fused kernel below instead and the
// update keeps r and A P (k_update_tma).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "small.cuh"
#include "spmv.cuh"

namespace sscg {

namespace {

// One level of the matrix-powers kernel (Algorithm 4): y = A u_j, written to
// AU_j when au_out != null; u_{j+1} = B^-1 y (when u_next != null; B^-1 the
// array dinv, or the constant dinv_c when dinv is null and dinv_c != 0, or
// none); the matrix in CSR tiles or, with DM != 0, its diagonal form (mode DM of
// spmv_dia_df for double-float); moment partials
// mu_{2j+1} = u_j . y and mu_{2j+2} = y . B^-1 y.  With `last` set, the last
// CTA reduces mu_1..mu_{2s-1} and runs Algorithm 6.
template <class A, int VM, int DM>
__global__ void __launch_bounds__(kThreads, dia_min_blocks<A, DM>()) k_level(MatView M, const typename A::S* __restrict__ dinv,
                                                    double dinv_c, const typename A::S* __restrict__ u_in,
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
    const R dc = A::from_d(dinv_c);
    auto xf = [&](int c) { return A::ldg(u_in + c); };
    auto epi = [&](int row, R y) {
        if (au_out) A::st(au_out + row, y);
        m1 = A::fma(A::ldg(u_in + row), y, m1);
        if (u_next || want_m2) {
            R z = dinv ? A::mul(A::ld(dinv + row), y) : (dinv_c != 0.0 ? A::mul(dc, y) : y);
            if (u_next) A::st(u_next + row, z);
            m2 = A::fma(y, z, m2);
        }
    };
    bool ok = true;
    if constexpr (DM >= 7 && A::kind == 0) {
        // Diagonal form, Laplacian class, FP64 (spmv_dia_lap_f64): with the
        // neighbour sum S, u_{j+1} = u + (c_off / d) S under Jacobi (B^-1 the
        // constant 1/d) and c_centre u + c_off S without a preconditioner;
        // mu_{2j+1} = u . A u = d sum u u_{j+1} and mu_{2j+2} = d sum u_{j+1}^2
        // (d = 1 without a preconditioner): three FP64 operations a row beyond
        // the sum, the moments' scale applied once per thread.
        const double cc = M.dc[DM / 2], co = (double)M.dco;
        const bool jac = dinv_c != 0.0;
        const double cz = co * dinv_c, ds = jac ? cc : 1.0;
        double a1 = 0.0, a2 = 0.0;
        auto run = [&](auto zf, auto m2on) {
            spmv_dia_lap_f64<DM>(M, u_in, [&](int i, double S, double xc) {
                const double z = zf(S, xc);
                u_next[i] = z;
                a1 = fma(xc, z, a1);
                if (decltype(m2on)::value) a2 = fma(z, z, a2);
            });
        };
        if (jac) {
            auto zf = [&](double S, double xc) { return fma(S, cz, xc); };
            if (want_m2) run(zf, std::true_type{});
            else run(zf, std::false_type{});
        } else {
            auto zf = [&](double S, double xc) { return fma(co, S, cc * xc); };
            if (want_m2) run(zf, std::true_type{});
            else run(zf, std::false_type{});
        }
        m1 = ds * a1;
        m2 = ds * a2;
    } else if constexpr (DM != 0 && A::kind == 1) {
        // Diagonal form (double-float): B^-1 is the constant dinv_c (Jacobi) or
        // the identity (dinv_c = 0), the level always writes u_{j+1} and never
        // AU_j.  Rows come in pairs; the moments are running Dot2 sums,
        // renormalised once per pair, with mu_{2j+2} = dinv_c * (y . y).
        const df64 d1c = dinv_c != 0.0 ? dc : df_make(1.f, 0.f);
        DotAcc d1{0.f, 0.f}, d2{0.f, 0.f};
        spmv_dia_df<DM>(M, u_in, [&](int i, df64 y0, df64 x0, df64 y1, df64 x1, bool has1) {
            const df64 z0 = df_mul(d1c, y0), z1 = df_mul(d1c, y1);
            if (has1) st_pair(u_next + i, z0, z1);
            else A::st(u_next + i, z0);
            dot_add(d1, x0, y0);
            dot_add(d1, x1, y1);
            dot_add_sq(d2, y0);
            dot_add_sq(d2, y1);
            dot_renorm(d1);
            dot_renorm(d2);
        });
        m1 = dot_value(d1);
        m2 = df_mul(d1c, dot_value(d2));
    } else if constexpr (DM != 0) {
        spmv_dia<A>(M, xf, epi);
    } else {
        ok = spmv_pipe<A, VM, kStages>(M, smem, xf, epi, ctrl);
    }
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

// Fused matrix-powers kernel: levels j0 .. j0+F-1 of one outer step in one
// launch, so the matrix is read from HBM about once per F levels.
//
// Work items are (level jl, tile t) pairs.  Item q has key q / F and level
// q % F, tile = key - jl * D.  Level jl of tile t needs level jl-1 of tiles
// t-h .. t+h (h: the matrix bandwidth in tiles), whose keys are at most
// key - (D - h); CTAs claim items from a global counter in increasing q, so
// every dependency is claimed before the item that needs it and the
// smallest unfinished item can always proceed.  D = h + 1 + (items in flight
// per level) keeps dependencies already finished when an item starts, and
// the rows a level re-reads (matrix rows, the previous level's vector) were
// touched D keys earlier: they are still in L2.  Each CTA prefetches its
// next item's matrix tile by bulk copy while computing the current one.
// A finished tile publishes flag[jl][t] = epoch (release store after a
// fence); consumers poll the flags with relaxed gpu-scope loads, fence, and
// read vectors produced in this launch through L2 (ld.global.cg).  Every wait is bounded by %globaltimer.
constexpr int kMaxFuse = 4;

// Flags are polled with relaxed gpu-scope loads (coherent at L2); one fence
// after the last flag orders the reads that follow.
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kFuseStages = 2;
constexpr int kFuseThreads = kThreads + 32;  // 8 consumer warps + 1 producer warp
constexpr int kFuseWarps = kThreads / 32;    // arrivals per finished tile
constexpr unsigned kNoItem = 0xffffffffu;

template <int VM>
__host__ __device__ constexpr size_t fused_smem(int cap) {
    return 64 + (size_t)kFuseStages * pipe_stage_bytes<VM>(cap);
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Counters: cnt[jl][t] gains one arrival from each consumer warp that has
// written its 32 rows of tile t at level slot jl.  want[jl] is the count a
// tile of slot jl reaches once this launch has finished it (the host adds
// kFuseWarps per launch that uses the slot; counters are zeroed per solve).
struct FuseWant {
    unsigned w[kMaxFuse];
};

template <class A, int VM>
__global__ void __launch_bounds__(kFuseThreads) k_mpk_fused(MatView M, const typename A::S* __restrict__ dinv,
                                                            typename A::S* __restrict__ blk, int ldn, int s, int j0,
                                                            int F, int T, int h, int D,
                                                            unsigned* __restrict__ cnt, FuseWant want,
                                                            double* __restrict__ part, int step, int last,
                                                            Ctrl* ctrl) {
    using R = typename A::R;
    using S = typename A::S;
    if (ctrl_done(ctrl)) return;
    extern __shared__ __align__(16) char smem_raw[];
    char* smem = align128(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);  // [kFuseStages]
    uint64_t* empty = full + kFuseStages;                 // [kFuseStages]
    char* stage0 = smem + 64;
    const size_t sb = pipe_stage_bytes<VM>(M.cap);
    __shared__ unsigned s_item[kFuseStages];
    __shared__ double red[2 * kMaxFuse * 16];
    const size_t ld = (size_t)ldn;
    const unsigned Q = (unsigned)(T + (F - 1) * D) * (unsigned)F;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto tile_of = [&](unsigned q, int& jl) {
        jl = (int)(q % (unsigned)F);
        return (int)(q / (unsigned)F) - jl * D;
    };
    if (threadIdx.x == 0) {
        for (int q = 0; q < kFuseStages; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kFuseWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    R m1[kMaxFuse], m2[kMaxFuse];
#pragma unroll
    for (int q = 0; q < kMaxFuse; q++) m1[q] = m2[q] = A::zero();
    bool ok = true;
    if (warp == kFuseWarps) {
        // producer: claim items in order and stage each one's matrix tile
        if (lane == 0) {
            for (int k = 0;; k++) {
                const int st = k % kFuseStages;
                if (k >= kFuseStages && !mbar_wait(&empty[st], (unsigned)((k / kFuseStages) - 1) & 1u)) {
                    ok = false;
                    break;
                }
                const unsigned q = atomicAdd(&ctrl->claim, 1u);
                int jl = 0, t = -1;
                if (q < Q) t = tile_of(q, jl);
                const bool live = q < Q && t >= 0 && t < T;
                s_item[st] = q < Q ? (live ? q : kNoItem - 1) : kNoItem;
                if (live) issue_tile<VM>(M, stage0 + (size_t)st * sb, &full[st], t);
                else mbar_arrive(&full[st]);  // nothing to copy: the phase completes on arrival
                if (q >= Q) break;
            }
        }
        __syncwarp();
    } else {
        // consumer warps run independently: no CTA barrier per item
        for (int k = 0;; k++) {
            const int st = k % kFuseStages;
            if (!mbar_wait(&full[st], (unsigned)(k / kFuseStages) & 1u)) {
                ok = false;
                break;
            }
            const unsigned cur = s_item[st];
            if (cur == kNoItem) break;
            if (cur != kNoItem - 1) {
                int jl;
                const int t = tile_of(cur, jl);
                if (jl > 0) {  // previous level's tiles t-h .. t+h complete?
                    const unsigned* c0 = cnt + (size_t)(jl - 1) * T;
                    const unsigned target = want.w[jl - 1];
                    const int lo = max(0, t - h), hi = min(T - 1, t + h);
                    bool dep_ok = true;
                    uint64_t t0 = 0;
                    for (int c = lo + lane; c <= hi && dep_ok; c += 32) {
                        unsigned spins = 0;
                        while (ld_relaxed_u32(c0 + c) < target) {
                            if (t0 == 0) t0 = globaltimer();
                            if ((++spins & 63u) == 0 && globaltimer() - t0 > kWaitLimitNs) {
                                dep_ok = false;
                                break;
                            }
                        }
                    }
                    dep_ok = __all_sync(0xffffffffu, dep_ok);
                    if (!dep_ok) {
                        if (lane == 0) {
                            ctrl->status = 3;  // SSCG_TIMEOUT
                            __threadfence();
                            atomicExch(&ctrl->done, 1);
                        }
                        ok = false;
                        break;
                    }
                    fence_acq_rel_gpu();  // the gathers below follow the observed counters
                }
                const int j = j0 + jl;
                const S* uj = blk + (size_t)j * ld;
                S* au = blk + (size_t)(s + j) * ld;
                S* un = (j + 1 < s) ? blk + (size_t)(j + 1) * ld : nullptr;
                const bool want_m2 = 2 * j + 2 <= 2 * s - 1;
                const bool fresh = jl > 0;  // u_j produced in this launch: read through L2
                compute_tile<A, VM>(
                    M, stage0 + (size_t)st * sb, t,
                    [&](int c) { return fresh ? A::ldcg(uj + c) : A::ldg(uj + c); },
                    [&](int row, R y) {
                        A::st(au + row, y);
                        R u = fresh ? A::ldcg(uj + row) : A::ldg(uj + row);
                        R a1 = A::mul(u, y), a2 = A::zero();
                        if (un || want_m2) {
                            R z = dinv ? A::mul(A::ld(dinv + row), y) : y;
                            if (un) A::st(un + row, z);
                            a2 = A::mul(y, z);
                        }
#pragma unroll
                        for (int q = 0; q < kMaxFuse; q++)
                            if (q == jl) {
                                m1[q] = A::add(m1[q], a1);
                                m2[q] = A::add(m2[q], a2);
                            }
                    });
                __syncwarp();  // the warp's rows are written
                if (lane == 0) red_release_add(cnt + (size_t)jl * T + t, 1u);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
    }
    if (!__syncthreads_and(ok)) return;
    const int G = gridDim.x;
#pragma unroll
    for (int q = 0; q < kMaxFuse; q++) {
        if (q >= F) break;
        R v[2] = {m1[q], m2[q]};
        double out[2];
        block_sum<A, 2>(v, red, out);
        if (threadIdx.x == 0) {
            part[(2 * (j0 + q)) * G + blockIdx.x] = out[0];
            part[(2 * (j0 + q) + 1) * G + blockIdx.x] = out[1];
        }
    }
    if (!last_cta(&ctrl->ticket[1])) return;
    if (threadIdx.x == 0) ctrl->claim = 0u;  // every CTA has left the claim loop
    if (!last) return;
    cta_sum_rows(part, 2 * s - 1, G, [&](int e, double v) { ctrl->mu[e + 1] = v; });
    SmallScratch* sc = reinterpret_cast<SmallScratch*>(smem);
    if (threadIdx.x < 32) {
        int st = warp_sw_monomial(ctrl, s, step, sc);
        if (threadIdx.x == 0 && st != 0) {
            ctrl->status = st;
            ctrl->done = 1;
        }
    }
}

// Fusion plan: levels per launch F, key lag D; F = 0 (one launch per level)
// unless SSCG_FUSED_MPK is set and the levels a launch would keep in L2 fit
// the budget.  Measured on GB300 the fused kernel cuts DRAM traffic 2.5x
// but is limited by item latency and dependency waits, so it is opt-in.
struct FusePlan {
    int F, T, h, D;
};

inline FusePlan plan_fusion(const sscg_mat* mat, int s, int G, unsigned flags) {
    FusePlan p{0, 0, 0, 0};
    if (!(flags & SSCG_FUSED_MPK)) return p;
    p.T = (int)((mat->n + kTileRows - 1) / kTileRows);
    p.h = (int)((mat->bandwidth + kTileRows - 1) / kTileRows);
    const double row_bytes = (4.0 + (double)mat->nnz / (double)mat->n * 8.0) + 48.0;
    for (int F = std::min(s, kMaxFuse); F >= 2; F--) {
        // items in flight: kFuseStages + 1 per CTA; lag them by 1.25x that many keys
        const int D = p.h + 1 + (5 * G * (kFuseStages + 1) / 4 + F - 1) / F + 8;
        const double l2 = (double)(F - 1) * D * kTileRows * row_bytes;
        if (l2 <= 72.0e6 && D < p.T) {
            p.F = F;
            p.D = D;
            return p;
        }
    }
    return p;
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
    unsigned* flags;
    void* xw;
    double* bdev;
    double* xdev;
    size_t bytes;
};

Layout plan(const sscg_mat* mat, const sscg_opts* o, int G, void* base, size_t cap) {
    Layout L{};
    L.ldn = (int64_t)align_up((size_t)mat->n, 64);
    L.G = G;
    Carve c(base, cap);
    L.ctrl = c.take<Ctrl>(1);
    L.hist = c.take<double>((size_t)o->maxit + 2);
    L.part = c.take<double>((size_t)G * (2 * kMaxS + 4));
    size_t blk = (size_t)L.ldn * (2 * o->s + 1);
    // margins around the blocks: the diagonal-form levels gather columns
    // 0..s-1 at indices down to -max|offset| without clamping
    const size_t g = dia_margin(mat);
    if (g) c.take<double>(g);
    L.blk[0] = c.take<double>(blk);
    if (g) c.take<double>(g);
    L.blk[1] = c.take<double>(blk);
    if (g) c.take<double>(g);
    L.r = c.take<double>((size_t)L.ldn);
    L.flags = c.take<unsigned>((size_t)kMaxFuse * ((mat->n + kTileRows - 1) / kTileRows));
    L.xw = (o->arith == SSCG_ARITH_F64) ? nullptr : c.take<double>((size_t)L.ldn);
    if (o->flags & SSCG_HOST_VECTORS) {
        L.bdev = c.take<double>((size_t)L.ldn);
        L.xdev = c.take<double>((size_t)L.ldn);
    }
    L.bytes = c.used;
    return L;
}

// Grid of k_update_fix for the block size s (1..6): its occupancy, with its
// two row buffers of shared memory, times the SMs; 0 when the attribute is refused.
template <int S>
inline int update_fix_grid_s(sscg_ctx* ctx, int64_t n) {
    if (cudaFuncSetAttribute(k_update_fix<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fix_row_smem<S>()) != cudaSuccess)
        return 0;
    return occupancy_grid(ctx, k_update_fix<S>, fix_row_smem<S>(), n);
}

inline int update_fix_grid(sscg_ctx* ctx, int s, int64_t n) {
    switch (s) {
        case 1: return update_fix_grid_s<1>(ctx, n);
        case 2: return update_fix_grid_s<2>(ctx, n);
        case 3: return update_fix_grid_s<3>(ctx, n);
        case 4: return update_fix_grid_s<4>(ctx, n);
        case 5: return update_fix_grid_s<5>(ctx, n);
        case 6: return update_fix_grid_s<6>(ctx, n);
        default: return 0;
    }
}

inline void launch_update_fix(int s, int grid, int64_t n, int ldn, double* blk_new, double* blk_old, double* x,
                              const double* diag, double diag_c, double* part, Ctrl* ctrl, double* hist,
                              cudaStream_t st) {
    const int N = (int)n;
    switch (s) {
        case 1: k_update_fix<1><<<grid, kThreads, fix_row_smem<1>(), st>>>(N, ldn, blk_new, blk_old, x, diag, diag_c, part, ctrl, hist); break;
        case 2: k_update_fix<2><<<grid, kThreads, fix_row_smem<2>(), st>>>(N, ldn, blk_new, blk_old, x, diag, diag_c, part, ctrl, hist); break;
        case 3: k_update_fix<3><<<grid, kThreads, fix_row_smem<3>(), st>>>(N, ldn, blk_new, blk_old, x, diag, diag_c, part, ctrl, hist); break;
        case 4: k_update_fix<4><<<grid, kThreads, fix_row_smem<4>(), st>>>(N, ldn, blk_new, blk_old, x, diag, diag_c, part, ctrl, hist); break;
        case 5: k_update_fix<5><<<grid, kThreads, fix_row_smem<5>(), st>>>(N, ldn, blk_new, blk_old, x, diag, diag_c, part, ctrl, hist); break;
        case 6: k_update_fix<6><<<grid, kThreads, fix_row_smem<6>(), st>>>(N, ldn, blk_new, blk_old, x, diag, diag_c, part, ctrl, hist); break;
        default: break;
    }
}

template <class A, int VM, int SB, int DM>
int run_sstep(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
              const Layout& L, const typename A::S* dinv, const typename A::S* diag, Ctrl* hctrl, Prof& P) {
    using S = typename A::S;
    constexpr bool DIA = DM != 0;
    cudaStream_t st = ctx->stream;
    const int n = (int)mat->n, s = o->s, G = L.G;
    const int cap = stage_cap(mat);
    MatView M = mat_view(mat);
    const size_t smem = std::max(stage_bytes<A, VM>(cap), sizeof(SmallScratch));
    const size_t smem_pipe = std::max(pipe_bytes<VM, kStages>(cap), sizeof(SmallScratch)) + 128;
    const size_t smem64 = stage_bytes<ArithF64, VAL_F64>(cap);
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_init<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // the diagonal form stages nothing; the last level's solves still use the scratch
    const size_t smem_lv = DIA ? sizeof(SmallScratch) + 128 : smem_pipe;
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_level<A, VM, DM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_lv));
    // with the diagonal form and Jacobi, D is the constant diagonal value
    const bool cd = DIA && dinv != nullptr;
    const typename A::S* dinv_l = cd ? nullptr : dinv;
    const typename A::S* diag_u = cd ? nullptr : diag;
    const double dinv_c = cd ? mat->dia_dinv : 0.0, diag_c = cd ? mat->dia_d : 0.0;
    const size_t smem_fused = std::max(fused_smem<VM>(cap), sizeof(SmallScratch)) + 128;
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_mpk_fused<A, VM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_fused));
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_true_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64));
    S* blk[2] = {(S*)L.blk[0], (S*)L.blk[1]};
    S* r = (S*)L.r;
    S* xw = A::kind == 0 ? (S*)x : (S*)L.xw;
    const size_t ld = (size_t)L.ldn;

    P.begin();
    const int Gi = occupancy_grid(ctx, k_init<A, VM>, smem, n);
    const int Gl = occupancy_grid(ctx, k_level<A, VM, DM>, smem_lv, n);
    int per_sm = 0;
    SSCG_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mpk_fused<A, VM>, kFuseThreads,
                                                                 smem_fused));
    const int Gf = std::max(1, std::min(kMaxGrid, ctx->sm_count * std::max(per_sm, 1)));
    const FusePlan fp = plan_fusion(mat, s, Gf, o->flags);
    if (fp.F > 0) SSCG_CUDA(ctx, cudaMemsetAsync(L.flags, 0, sizeof(unsigned) * kMaxFuse * fp.T, st));
    FuseWant want{};  // arrivals each level slot's counters reach after the current launch
    size_t smem_upd = 0;
    int Gu = 0;
    if (int e = update_tma_setup<A, SB>(ctx, n, s, &smem_upd, &Gu)) return e;
    size_t smem_updq = 0;
    int Gq = 0;
    if (int e = update_q_setup<A, SB>(ctx, n, s, &smem_updq, &Gq)) return e;
    // FP64 at s <= 6: P and Q as fixed-point dot products from the second step on
    const bool fix_upd = A::kind == 0 && s + 1 <= kFixMaxTerms && !(o->flags & SSCG_FMA_UPDATE);
    const int Gx = fix_upd ? update_fix_grid(ctx, s, n) : 0;
    if (fix_upd && Gx == 0)
        return set_err(ctx, SSCG_ERR_CUDA, "shared memory for the fixed-point block update refused");
    const int Gt = occupancy_grid(ctx, k_true_res, smem64, n);
    k_init<A, VM><<<Gi, kThreads, smem, st>>>(M, dinv, b, x, A::kind == 0 ? nullptr : xw, r, blk[0], L.part,
                                              L.ctrl, L.hist);
    P.end(FAM_INIT, 0);
    SSCG_CUDA(ctx, cudaGetLastError());

    const int per_chunk = std::max(1, 32 / (s + 1));
    ChunkPoll poll;
    SSCG_CUDA(ctx, poll.init());
    int launched = 0;
    int err = 0;
    while (launched < o->maxit) {
        int c = std::min(per_chunk, o->maxit - launched);
        for (int q = 0; q < c; q++) {
            const int k = launched + q;
            S* bn = blk[k & 1];
            S* bo = blk[(k + 1) & 1];
            if (fp.F > 0) {
                for (int j0 = 0; j0 < s; j0 += fp.F) {
                    const int F = std::min(fp.F, s - j0);
                    for (int q = 0; q < F; q++) want.w[q] += kFuseWarps;
                    P.begin();
                    k_mpk_fused<A, VM><<<Gf, kFuseThreads, smem_fused, st>>>(M, dinv, bn, (int)L.ldn, s, j0, F, fp.T,
                                                                            fp.h, fp.D, L.flags, want, L.part, k,
                                                                            j0 + F == s, L.ctrl);
                    P.end(FAM_MPK, k);
                }
            } else {
                // u_{j+1} = D^-1 A u_j into column j+1 (all j, u_{s+1} too); A u_j is not stored
                for (int j = 0; j < s; j++) {
                    P.begin();
                    k_level<A, VM, DM><<<Gl, kThreads, smem_lv, st>>>(M, dinv_l, dinv_c, bn + j * ld, nullptr,
                                                                     bn + (j + 1) * ld, L.part, j, s, k, j == s - 1,
                                                                     L.ctrl);
                    P.end(FAM_MPK, k);
                }
            }
            P.begin();
            if (fp.F > 0)
                k_update_tma<A, SB><<<Gu, kUpdRows, smem_upd, st>>>(n, (int)L.ldn, s, bn, bo, xw, r, dinv, L.part,
                                                                    k == 0, 1, L.ctrl, L.hist);
            else if constexpr (A::kind == 0) {
                if (fix_upd && k > 0)
                    launch_update_fix(s, Gx, n, (int)L.ldn, bn, bo, xw, diag_u, diag_c, L.part, L.ctrl, L.hist, st);
                else
                    k_update_q<A, SB><<<Gq, kThreads, 0, st>>>(n, (int)L.ldn, s, bn, bo, xw, diag_u, diag_c,
                                                               L.part, k == 0, L.ctrl, L.hist);
            } else
                k_update_q<A, SB><<<Gq, kThreads, 0, st>>>(n, (int)L.ldn, s, bn, bo, xw, diag_u, diag_c,
                                                           L.part, k == 0, L.ctrl, L.hist);
            P.end(FAM_UPDATE, k);
        }
        if (cudaGetLastError() != cudaSuccess) { err = 1; break; }
        launched += c;
        int fin = 0;
        cudaError_t pe = cudaSuccess;
        const bool got = poll.step(ctx->pinned, &L.ctrl->done, st, &fin, &pe);
        SSCG_CUDA(ctx, pe);
        if (got && fin) break;
    }
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

// The update kernels are built for block sizes up to 4, 8 and 16.
template <class A, int VM, int DM>
int run_sstep_sb(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* o,
                 const Layout& L, const typename A::S* dinv, const typename A::S* diag, Ctrl* hctrl, Prof& P) {
    if (o->s <= 4) return run_sstep<A, VM, 4, DM>(ctx, mat, b, x, o, L, dinv, diag, hctrl, P);
    if (o->s <= 8) return run_sstep<A, VM, 8, DM>(ctx, mat, b, x, o, L, dinv, diag, hctrl, P);
    return run_sstep<A, VM, 16, DM>(ctx, mat, b, x, o, L, dinv, diag, hctrl, P);
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
    // the diagonal form serves the sequential levels (the fused kernel stages CSR tiles)
    const bool dia = mat->dia && !(o->flags & SSCG_FUSED_MPK);
    int rc;
    const int s = o->s;
    Prof* prof = new Prof(ctx, (o->flags & SSCG_PROFILE) != 0);
    if (!prof->reserve((int)std::min<int64_t>(65536, (int64_t)o->maxit * (s + 1) + 64))) {
        delete prof;
        return set_err(ctx, SSCG_ERR_CUDA, "could not create profiling events");
    }
    if (o->arith == SSCG_ARITH_F64) {
        const double* dinv = jac ? mat->dinv : nullptr;
        const double* diag = jac ? mat->diag : nullptr;
        // plan() carves margins around both blocks whenever the matrix has the diagonal form
        const int dm = dia ? dia_mode(mat, true) : 0;
        if (dm == 7) rc = run_sstep_sb<ArithF64, VAL_F64, 7>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else if (dm == 27) rc = run_sstep_sb<ArithF64, VAL_F64, 27>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else if (dm != 0) rc = run_sstep_sb<ArithF64, VAL_F64, 1>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else rc = run_sstep_sb<ArithF64, VAL_F64, 0>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
    } else {
        const float2* dinv = jac ? mat->dinv_df : nullptr;
        const float2* diag = jac ? mat->diag_df : nullptr;
        // plan() carves margins around both blocks whenever the matrix has the diagonal form
        const int dm = dia ? dia_mode(mat, true) : 0;
        if (dm == 7) rc = run_sstep_sb<ArithDF64, VAL_F32, 7>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else if (dm == 27) rc = run_sstep_sb<ArithDF64, VAL_F32, 27>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else if (dm != 0) rc = run_sstep_sb<ArithDF64, VAL_F32, 2>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else if (mat->exact_fp32) rc = run_sstep_sb<ArithDF64, VAL_F32, 0>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
        else rc = run_sstep_sb<ArithDF64, VAL_DF, 0>(ctx, mat, bd, xd, o, L, dinv, diag, &h, *prof);
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
