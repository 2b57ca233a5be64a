// Batched s-step CG: many independent SPD systems, each with 1..8 right-hand
// sides, solved by one persistent cooperative kernel.
//
// Every system runs Algorithm 3 with the monomial basis, the Jacobi
// preconditioner and the moment recurrence of Algorithm 6, per right-hand
// side, as the single-system path does.  The kernel walks the phases of an
// outer step for all systems at once, separated by grid-wide barriers:
//
//   level j = 0..s-1   matrix-powers level (Algorithm 4) of every active
//                      system: U_{j+1} = D^-1 A U_j for all its right-hand
//                      sides in one pass over the matrix (SpMM; CSR, or the
//                      constant-coefficient diagonal form for stencils),
//                      moment partials mu_{2j+1}, mu_{2j+2} per item
//   solve              per system (one CTA): reduce the partials, test
//                      convergence, run Algorithm 6 per right-hand side
//                      (one warp each)
//   update             block updates of Algorithm 3 in the z = D^-1 r,
//                      Q = D^-1 A P form (A U is never stored, as in the
//                      single-system path) and the partials of ||r||^2 and
//                      mu_0 for the next step
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
// Per-phase level kernel: CSR entries of a 256-row sub-tile staged in shared
// memory (column index + value as hi/lo floats or a double: 12 bytes).
constexpr int kLevelCap = 3072;
constexpr size_t kLevelSmem = (size_t)(kBThreads + 4) * 4 + (size_t)kLevelCap * 12 + 64;

enum SysState { SYS_ACTIVE = 0, SYS_EXPORT = 1, SYS_FINISHED = 2 };

struct BSys {
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    const float* vhi;
    const float* vlo;
    const void* dinv;  // 1/diag: double (F64) or float2 (double-float); null: the constant dinv_c
    const void* diag;  // diag, the same way (constant diag_c)
    void* blk[2];      // 2s+1 columns of n x R each: U_1..U_{s+1} | Q; P overwrites U_1..U_s
    void* xw;          // correction to x0, n x R
    double* lpart;     // (2s-1) R rows of `items` moment partials
    double* upart;     // 3 R rows: ||r||^2, mu_0, ||b||^2 (step 0) / true residual^2
    const uint32_t* dmask;  // constant-coefficient diagonal form (dk > 0), else CSR
    int dk, pad0;
    int doff[kDiaMax];
    float dcf[kDiaMax];
    int dcen, dlap;  // index of offset 0; every off-centre value equals dco
    float dco, pad1;
    double dinv_c, diag_c;
    int n, R, exact, T;
    int items, item0, rhs0, pad;
};

// The per-row fields of a system, copied into registers once per item (the
// loops below store to global memory, so fields read through the BSys
// reference would be reloaded on every element).
struct BReg {
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    const float* vhi;
    const float* vlo;
    const uint32_t* dmask;
    const void* dinv;
    const void* diag;
    double dinv_c, diag_c;
    int n, R, exact, dk;
    int dcen, dlap;
    float dco;
};

__device__ __forceinline__ BReg breg(const BSys& y) {
    BReg b;
    b.rowptr = y.rowptr;
    b.col = y.col;
    b.val = y.val;
    b.vhi = y.vhi;
    b.vlo = y.vlo;
    b.dmask = y.dmask;
    b.dinv = y.dinv;
    b.diag = y.diag;
    b.dinv_c = y.dinv_c;
    b.diag_c = y.diag_c;
    b.n = y.n;
    b.R = y.R;
    b.exact = y.exact;
    b.dk = y.dk;
    b.dcen = y.dcen;
    b.dlap = y.dlap;
    b.dco = y.dco;
    return b;
}

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
    int skip_cta;             // fault injection: this CTA skips its first barrier arrival (-1: none)
    unsigned long long wait_ns;  // limit of every barrier wait
    int fma_update;           // FP64 at s = 4: P and Q by FP64 FMAs instead of fixed-point dot products
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
// false when the kernel must stop (a wait expired here or elsewhere).  Every
// wait gives up after wait_ns.  With skip_cta set (fault injection for tests
// of the bounded waits), that CTA does not arrive: the others' waits expire
// and set SSCG_TIMEOUT, while it waits (bounded as well) for that error and
// returns; the barrier's counters are reset by the next solve.
__device__ bool grid_sync(GCtl* g, int skip_cta, unsigned long long wait_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x == skip_cta) {
        const uint64_t t0 = globaltimer();
        while (!*(volatile int*)&g->err) {
            if (globaltimer() - t0 > 2 * wait_ns + 100000000ull) {
                atomicCAS(&g->err, 0, SSCG_TIMEOUT);
                break;
            }
            __nanosleep(1000);
        }
        s_ok = 0;
    } else if (threadIdx.x == 0) {
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
                if (globaltimer() - t0 > wait_ns) {
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

    static __device__ __forceinline__ Rv dinv_of(const BReg& y, int i) {
        return y.dinv ? A::ldg(reinterpret_cast<const S*>(y.dinv) + i) : A::from_d(y.dinv_c);
    }

    static __device__ __forceinline__ Rv diag_of(const BReg& y, int i) {
        return y.diag ? A::ldg(reinterpret_cast<const S*>(y.diag) + i) : A::from_d(y.diag_c);
    }

    // (A v_r)[i] for right-hand side r of the interleaved vectors v.  The R
    // threads of a row read the same matrix entries (broadcast through L1);
    // their gathers are contiguous.  RO: v was written by an earlier launch
    // (read-only path); otherwise through L2.  soff/scf: the diagonal form's
    // offsets and values in shared memory.
    template <bool RO, bool LAP = true, bool LAP27 = false>
    static __device__ __forceinline__ Rv spmv_elem(const BReg& y, const int* soff, const float* scf, int i, int r,
                                                   const S* v) {
        const int R = y.R;
        Rv acc = A::zero();
        if (y.dk) {
            const uint32_t m = __ldg(y.dmask + i);
            if constexpr (A::kind == 1 && LAP) {
                if (y.dlap) {
                    // Laplacian class: the present neighbours summed as
                    // double-float values (TwoSum of the high parts, low parts
                    // and errors in a second float), scaled once by their
                    // common value, then the centre by one Dot2 step
                    float sh = 0.f, se = 0.f;
                    auto nb = [&](int t) {
                        if (t == y.dcen || !((m >> t) & 1u)) return;
                        const S* px = v + (size_t)(i + soff[t]) * R + r;
                        const Rv x = RO ? A::ldg(px) : A::ldcg(px);
                        float u, w;
                        two_sum(sh, x.hi, u, w);
                        sh = u;
                        se = __fadd_rn(se, __fadd_rn(w, x.lo));
                    };
                    if (y.dk == 7) {
#pragma unroll
                        for (int t = 0; t < 7; t++) nb(t);
                    } else {
                        for (int t = 0; t < y.dk; t++) nb(t);
                    }
                    const S* pc = v + (size_t)i * R + r;
                    const Rv xc = RO ? A::ldg(pc) : A::ldcg(pc);
                    const float co = y.dco, p = __fmul_rn(co, sh);
                    Dot2Acc d{p, __fmaf_rn(co, se, __fmaf_rn(co, sh, -p))};
                    dot2_add(d, scf[y.dcen], xc);
                    return dot2_result(d);
                }
                Dot2Acc d{0.f, 0.f};
                for (int t = 0; t < y.dk; t++) {
                    if (!((m >> t) & 1u)) continue;
                    const S* px = v + (size_t)(i + soff[t]) * R + r;
                    dot2_add(d, scf[t], RO ? A::ldg(px) : A::ldcg(px));
                }
                return dot2_result(d);
            } else {
                if constexpr (A::kind == 0 && LAP) {
                    // FP64 7-point Laplacian class: the neighbour sum in fixed point on
                    // the integer units (lap_neighbour_sum), then one FMA with the centre
                    // (the 27-point rows keep the FMA loop below: their 26 fixed-point
                    // terms would triple this kernel's registers)
                    if (y.dlap && y.dk == 7 && y.dcen == 3) {
                        auto ld = [&](int t) {
                            const S* px = v + (size_t)(i + soff[t]) * R + r;
                            return RO ? A::ldg(px) : A::ldcg(px);
                        };
                        const double Sn = lap_neighbour_sum<7>(m, ld);
                        return ::fma((double)scf[3], ld(3), (double)y.dco * Sn);
                    }
                    // FP64 27-point Laplacian class: the 26 neighbours in fixed point
                    // (only in the level kernel of kind 3, built for 128 registers)
                    if constexpr (LAP27) {
                        if (y.dlap && y.dk == 27 && y.dcen == 13) {
                            auto ld = [&](int t) {
                                const S* px = v + (size_t)(i + soff[t]) * R + r;
                                return RO ? A::ldg(px) : A::ldcg(px);
                            };
                            const double Sn = lap_neighbour_sum<27>(m, ld);
                            return ::fma((double)scf[13], ld(13), (double)y.dco * Sn);
                        }
                    }
                }
                for (int t = 0; t < y.dk; t++) {
                    if (!((m >> t) & 1u)) continue;
                    const S* px = v + (size_t)(i + soff[t]) * R + r;
                    const Rv x = RO ? A::ldg(px) : A::ldcg(px);
                    if constexpr (A::kind == 1) acc = df_fma_f(x, scf[t], acc);
                    else acc = ::fma((double)scf[t], x, acc);
                }
            }
            return acc;
        }
        const int k0 = __ldg(y.rowptr + i), k1 = __ldg(y.rowptr + i + 1);
        for (int k = k0; k < k1; k++) {
            const S* px = v + (size_t)__ldg(y.col + k) * R + r;
            const Rv x = RO ? A::ldg(px) : A::ldcg(px);
            if constexpr (A::kind == 1) {
                if (y.exact) acc = df_fma_f(x, __ldg(y.vhi + k), acc);
                else acc = df_fma(x, df_make(__ldg(y.vhi + k), __ldg(y.vlo + k)), acc);
            } else {
                acc = ::fma(__ldg(y.val + k), x, acc);
            }
        }
        return acc;
    }

    // (A x_r)[i] for FP64 column-major user vectors X (n x R, column r at r n).
    static __device__ __forceinline__ Rv spmv_user_elem(const BReg& y, int i, int r, const double* X) {
        Rv acc = A::zero();
        const double* xr = X + (size_t)r * y.n;
        const int k0 = __ldg(y.rowptr + i), k1 = __ldg(y.rowptr + i + 1);
        for (int k = k0; k < k1; k++) {
            const int c = __ldg(y.col + k);
            Rv a;
            if constexpr (A::kind == 1) a = y.exact ? df_make(__ldg(y.vhi + k), 0.f) : df_make(__ldg(y.vhi + k), __ldg(y.vlo + k));
            else a = __ldg(y.val + k);
            acc = A::fma(a, A::from_d(__ldcg(xr + c)), acc);
        }
        return acc;
    }
};

// Sum over the CTA of the values of slot 0..ns-1 (a thread's value belongs
// to slot `slot`; slot >= ns contributes nothing), each by warp shuffles and
// then warps in a fixed order; thread q < ns receives slot q's sum.
template <class A>
__device__ __forceinline__ void cta_sum_slots(typename A::R val, int slot, int ns, double (*sh)[kBWarps],
                                              double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < ns; q++) {
        typename A::R w = warp_sum<A>(slot == q ? val : A::zero());
        if (lane == 0) sh[q][warp] = A::to_d(w);
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        double t = 0.0;
        for (int w = 0; w < kBWarps; w++) t += sh[threadIdx.x][w];
        *out = t;
    }
    __syncthreads();
}

// Work mapping inside an item of a system with R right-hand sides: thread t
// takes right-hand side r = t mod R of rows r0 + t / R, + 256 / R, ...
// (interleaved element i R + r), so a warp's loads of any column are
// contiguous and each thread keeps one accumulator per quantity.
#define ITEM_MAP(y)                                              \
    const BReg yb = breg(y);                                     \
    const int R = yb.R;                                          \
    const int rows_it = kBThreads / R;                           \
    const int tr = (int)threadIdx.x / R;                         \
    const int r = (int)threadIdx.x - tr * R;                     \
    const int slot = tr < rows_it ? r : kMaxR;                   \
    (void)slot

// Init phase: items it0, it0 + itstep, ... of every system.
template <class A>
__device__ void ph_init(const BArgs& a, int it0, int itstep) {
    using K = BK<A>;
    using Rv = typename A::R;
    using S = typename A::S;
    __shared__ double red[2 * kMaxR][kBWarps];
    // ---------------------------------------------------------- init
    // r = b - A x0, z = D^-1 r = U_1, correction 0; partials ||r||^2, mu_0, ||b||^2
    for (int it = it0; it < a.nitems; it += itstep) {
        const int k = __ldg(a.item_sys + it);
        const BSys& y = a.sys[k];
        ITEM_MAP(y);
        const int li = it - y.item0;
        const int r0 = li * y.T, r1 = min(y.n, r0 + y.T);
        const double* B = a.tuning ? nullptr : a.io[2 * k];
        const double* X = a.tuning ? nullptr : a.io[2 * k + 1];
        Rv rr = A::zero(), rz = A::zero(), bb = A::zero();
        const Rv dinv_cst = A::from_d(yb.dinv_c);
        S* u0 = K::col(y.blk[0], 0, y);
        S* xw = reinterpret_cast<S*>(y.xw);
        for (int i = r0 + tr; tr < rows_it && i < r1; i += rows_it) {
            const size_t o = (size_t)i * R + r;
            const Rv ax = X ? K::spmv_user_elem(yb, i, r, X) : A::zero();
            const double bv = B ? __ldg(B + (size_t)r * y.n + i) : splitmix_u(0xBA7C5EEDull + k, o);
            const Rv b = A::from_d(bv);
            const Rv res = A::sub(b, ax);
            const Rv z = A::mul(yb.dinv ? A::ldg(reinterpret_cast<const S*>(yb.dinv) + i) : dinv_cst, res);
            A::st(u0 + o, z);
            A::st(xw + o, A::zero());
            rr = A::fma(res, res, rr);
            rz = A::fma(res, z, rz);
            bb = A::fma(b, b, bb);
        }
        double out = 0.0;
        cta_sum_slots<A>(rr, slot, R, red, &out);
        if (threadIdx.x < R) y.upart[(size_t)threadIdx.x * y.items + li] = out;
        cta_sum_slots<A>(rz, slot, R, red, &out);
        if (threadIdx.x < R) y.upart[(size_t)(R + threadIdx.x) * y.items + li] = out;
        cta_sum_slots<A>(bb, slot, R, red, &out);
        if (threadIdx.x < R) y.upart[(size_t)(2 * R + threadIdx.x) * y.items + li] = out;
    }
}

// Level j of every active system (RO: u_j was written by an earlier launch,
// so the gathers may use the read-only path; inside one cooperative launch
// they go through L2).
// KIND: 0 every system; 1 CSR systems only; 2 diagonal-form systems only; 3
// FP64 27-point Laplacian-class diagonal-form systems only, which kind 2 then
// skips (the per-phase mode launches the kinds separately, so each keeps its
// own register budget: kind 3's fixed-point sum of 26 neighbours holds 128).
template <class A, bool RO, int KIND = 0>
__device__ void ph_level(const BArgs& a, int j, int it0, int itstep) {
    using K = BK<A>;
    using Rv = typename A::R;
    using S = typename A::S;
    __shared__ double red[2 * kMaxR][kBWarps];
    __shared__ int s_doff[kDiaMax];
    __shared__ float s_dcf[kDiaMax];
    const int s = a.s;
    for (int it = it0; it < a.nitems; it += itstep) {
        const int k = __ldg(a.item_sys + it);
        const BSys& y = a.sys[k];
        const int state = __ldcg(&a.bctl[k].state);
        if (state == SYS_FINISHED || (state == SYS_EXPORT && (j > 0 || a.tuning))) continue;
        // the other kernels' systems (kind 3: FP64 27-point Laplacian-class diagonal form)
        const bool lap27 = A::kind == 0 && y.dk == 27 && y.dlap && y.dcen == 13;
        if ((KIND == 1 && y.dk) || (KIND == 2 && (!y.dk || lap27)) || (KIND == 3 && !lap27)) continue;
        ITEM_MAP(y);
        const int li = it - y.item0;
        const int r0 = li * y.T, r1 = min(y.n, r0 + y.T);
        if (state == SYS_EXPORT) {
            // true residual of the exported x: b - A x
            const double* B = a.io[2 * k];
            const double* X = a.io[2 * k + 1];
            Rv tres = A::zero();
            for (int i = r0 + tr; tr < rows_it && i < r1; i += rows_it) {
                const Rv e = A::sub(A::from_d(__ldg(B + (size_t)r * yb.n + i)), K::spmv_user_elem(yb, i, r, X));
                tres = A::fma(e, e, tres);
            }
            double out = 0.0;
            cta_sum_slots<A>(tres, slot, R, red, &out);
            if (threadIdx.x < R) y.upart[(size_t)(2 * R + threadIdx.x) * y.items + li] = out;
            continue;
        }
        const int step = __ldcg(&a.bctl[k].step);
        void* blk = y.blk[step & 1];
        const S* uj = K::col(blk, j, y);
        S* un = K::col(blk, j + 1, y);  // u_{j+1} = D^-1 A u_j; A u_j is not stored
        const bool want_m2 = 2 * j + 2 <= 2 * s - 1;
        const Rv dinv_cst = A::from_d(yb.dinv_c);
        Rv m1 = A::zero(), m2 = A::zero();
        DotAcc d1{0.f, 0.f}, d2{0.f, 0.f};  // diagonal form, double-float: running Dot2 sums
        auto epi = [&](int i, Rv av) {
            const size_t o = (size_t)i * R + r;
            m1 = A::fma(RO ? A::ldg(uj + o) : A::ldcg(uj + o), av, m1);
            const Rv z = A::mul(yb.dinv ? A::ldg(reinterpret_cast<const S*>(yb.dinv) + i) : dinv_cst, av);
            A::st(un + o, z);
            if (want_m2) m2 = A::fma(av, z, m2);
        };
        auto epi_dia = [&](int i, Rv av) {
            if constexpr (A::kind == 1) {
                const size_t o = (size_t)i * R + r;
                const Rv ui = RO ? A::ldg(uj + o) : A::ldcg(uj + o);
                const Rv z = A::mul(dinv_cst, av);  // the diagonal form's D is constant
                A::st(un + o, z);
                dot_add(d1, ui, av);
                dot_add_sq(d2, av);  // av . D^-1 av = dinv_c (av . av), scaled below
                dot_renorm(d1);
                dot_renorm(d2);
            } else {
                epi(i, av);
            }
        };
        if (!RO || yb.dk) {
            if (yb.dk) {
                __syncthreads();  // the previous item is done with the offsets
                if (threadIdx.x < yb.dk) {
                    s_doff[threadIdx.x] = y.doff[threadIdx.x];
                    s_dcf[threadIdx.x] = y.dcf[threadIdx.x];
                }
                __syncthreads();
            }
            for (int i = r0 + tr; tr < rows_it && i < r1; i += rows_it) {
                if constexpr (KIND == 1) {
                    epi(i, K::template spmv_elem<RO, false>(yb, s_doff, s_dcf, i, r, uj));
                } else {
                    const Rv av = K::template spmv_elem<RO, true, KIND == 3>(yb, s_doff, s_dcf, i, r, uj);
                    if (yb.dk) epi_dia(i, av);
                    else epi(i, av);
                }
            }
        } else if constexpr (KIND != 2 && KIND != 3) {
            // CSR: stage each 256-row sub-tile's row pointers, column indices
            // and values in shared memory with coalesced loads; the R threads
            // of a row then read them from there
            extern __shared__ __align__(16) char lsm[];
            int* s_rp = reinterpret_cast<int*>(lsm);
            int* s_col = s_rp + kBThreads + 4;
            char* vbase = reinterpret_cast<char*>(s_col + kLevelCap);
            float2* s_vf = reinterpret_cast<float2*>(vbase);
            double* s_vd = reinterpret_cast<double*>(vbase);
            for (int t0 = r0; t0 < r1; t0 += kBThreads) {
                const int rows_t = min(kBThreads, r1 - t0);
                __syncthreads();  // the previous sub-tile is done with the buffers
                for (int q = threadIdx.x; q <= rows_t; q += kBThreads) s_rp[q] = __ldg(yb.rowptr + t0 + q);
                __syncthreads();
                const int base = s_rp[0];
                const int staged = min(s_rp[rows_t] - base, kLevelCap);
                for (int q = threadIdx.x; q < staged; q += kBThreads) {
                    s_col[q] = __ldg(yb.col + base + q);
                    if constexpr (A::kind == 1) s_vf[q] = make_float2(__ldg(yb.vhi + base + q), __ldg(yb.vlo + base + q));
                    else s_vd[q] = __ldg(yb.val + base + q);
                }
                __syncthreads();
                for (int rl = tr; tr < rows_it && rl < rows_t; rl += rows_it) {
                    const int ks = s_rp[rl] - base, ke = s_rp[rl + 1] - base;
                    Rv acc = A::zero();
                    for (int q = ks; q < ke; q++) {
                        const bool in = q < staged;
                        const int c = in ? s_col[q] : __ldg(yb.col + base + q);
                        const Rv x = A::ldg(uj + (size_t)c * R + r);
                        if constexpr (A::kind == 1) {
                            const float2 v = in ? s_vf[q] : make_float2(__ldg(yb.vhi + base + q), __ldg(yb.vlo + base + q));
                            acc = yb.exact ? df_fma_f(x, v.x, acc) : df_fma(x, df_make(v.x, v.y), acc);
                        } else {
                            acc = ::fma(in ? s_vd[q] : __ldg(yb.val + base + q), x, acc);
                        }
                    }
                    epi(t0 + rl, acc);
                }
            }
        }
        if constexpr (A::kind == 1) {
            if (yb.dk) {
                m1 = dot_value(d1);
                m2 = want_m2 ? df_mul(dinv_cst, dot_value(d2)) : A::zero();
            }
        }
        double out = 0.0;
        cta_sum_slots<A>(m1, slot, R, red, &out);
        if (threadIdx.x < R) y.lpart[(size_t)(2 * j * R + threadIdx.x) * y.items + li] = out;  // mu_{2j+1}
        if (want_m2) {
            cta_sum_slots<A>(m2, slot, R, red, &out);
            if (threadIdx.x < R) y.lpart[(size_t)((2 * j + 1) * R + threadIdx.x) * y.items + li] = out;
        }
    }
}

// Solve phase: systems k0, k0 + kstep, ..., one CTA each.
template <class A>
__device__ void ph_solve(const BArgs& a, int k0, int kstep) {
    __shared__ double sw_red[(2 * kMaxSB + 2) * kMaxR];
    __shared__ SmallScratchT<kMaxSB> scratch[kBWarps];
    const int s = a.s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = k0; k < a.nsys; k += kstep) {
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
            // four independent sums per lane keep four loads in flight
            double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
            int b = lane;
            for (; b + 96 < items; b += 128) {
                t0 += __ldcg(src + b);
                t1 += __ldcg(src + b + 32);
                t2 += __ldcg(src + b + 64);
                t3 += __ldcg(src + b + 96);
            }
            for (; b < items; b += 32) t0 += __ldcg(src + b);
            double t = (t0 + t1) + (t2 + t3);
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
            for (int q = 0; q < R; q++) all &= a.rc[y.rhs0 + q].done ? 1 : 0;
            if (all) bc->state = SYS_EXPORT;
            else bc->step = step + 1;
        }
        __syncthreads();
    }
}

// Update phase of every active (or exporting) system.
template <class A, int SB>
__device__ void ph_update(const BArgs& a, int it0, int itstep) {
    using K = BK<A>;
    using Rv = typename A::R;
    using S = typename A::S;
    __shared__ double red[2 * kMaxR][kBWarps];
    // alpha and beta converted once per item (a double-to-double-float
    // conversion runs on the FP64 pipe, 1/57 of the FP32 rate)
    __shared__ Rv s_alpha[kMaxR][kMaxSB];
    __shared__ Rv s_beta[kMaxR][kMaxSB * kMaxSB];
    __shared__ int s_act[kMaxR];
    // FP64 with s = SB <= 4: P and Q as fixed-point dot products (fixsum.cuh),
    // each right-hand side's coefficient columns aligned once per item
    constexpr bool kFix = A::kind == 0 && SB + 1 <= kFixMaxTerms;
    constexpr int FS = kFix ? SB : 1;
    __shared__ FixLimbs s_cf[kMaxR][FS][FS + 1];
    __shared__ int s_fc[kMaxR][FS];
    __shared__ int s_rng[kMaxR][2];
    const int s = a.s;
    for (int it = it0; it < a.nitems; it += itstep) {
        const int k = __ldg(a.item_sys + it);
        const BSys& y = a.sys[k];
        const int state = __ldcg(&a.bctl[k].state);
        if (state == SYS_FINISHED) continue;
        ITEM_MAP(y);
        const int li = it - y.item0;
        const int r0 = li * y.T, r1 = min(y.n, r0 + y.T);
        if (state == SYS_EXPORT) {
            if (a.tuning) continue;
            double* X = const_cast<double*>(a.io[2 * k + 1]);
            const S* xw = reinterpret_cast<const S*>(y.xw);
            const int zero = __ldcg(&a.rc[y.rhs0 + r].zero_rhs);
            for (int i = r0 + tr; tr < rows_it && i < r1; i += rows_it) {
                double* px = X + (size_t)r * y.n + i;
                *px = zero ? 0.0 : *px + A::to_d(A::ldcg(xw + (size_t)i * R + r));
            }
            continue;
        }
        const int kk = __ldcg(&a.bctl[k].step) - 1;  // the outer step being completed
        __syncthreads();
        for (int e = threadIdx.x; e < R * (s + s * s + 1); e += kBThreads) {
            const int rq = e / (s + s * s + 1), q = e % (s + s * s + 1);
            const Ctrl* c = &a.rc[y.rhs0 + rq];
            if (q < s) s_alpha[rq][q] = A::from_d(__ldcg(c->alpha + q));
            else if (q < s + s * s) s_beta[rq][q - s] = A::from_d(__ldcg(c->beta + (q - s)));
            else s_act[rq] = __ldcg(&c->done) ? 0 : 1;
        }
        __syncthreads();
        bool fixp = false;  // the same for every thread of the item
        if constexpr (kFix) {
            fixp = s == SB && kk > 0 && !a.fma_update;
            if (fixp) {
                for (int e = threadIdx.x; e < R * SB; e += kBThreads) {
                    const int rq = e / SB, j = e % SB;
                    s_fc[rq][j] = fix_coef_column<SB>(&s_beta[rq][0], j, s_cf[rq][j]);
                }
                __syncthreads();
                if (threadIdx.x < R) fix_row_range<SB>(s_fc[threadIdx.x], &s_rng[threadIdx.x][0], &s_rng[threadIdx.x][1]);
                __syncthreads();
            }
        }
        // z / Q form (Algorithm 3 multiplied by D^-1, as the single-system
        // path): P_j = U_j + sum P_old beta, Q_j = U_{j+1} + sum Q_old beta,
        // x += P alpha, z -= Q alpha; the next z goes to column 0 of the old block
        S* nb = reinterpret_cast<S*>(y.blk[kk & 1]);
        S* ob = reinterpret_cast<S*>(y.blk[(kk + 1) & 1]);
        const size_t nR = (size_t)y.n * R;
        S* xw = reinterpret_cast<S*>(y.xw);
        const bool act = s_act[r] != 0;
        const Rv dcst = A::from_d(yb.diag_c);
        Rv rr = A::zero(), rz = A::zero();
        for (int i = r0 + tr; tr < rows_it && i < r1; i += rows_it) {
            const size_t o = (size_t)i * R + r;
            if (!act) {
                A::st(ob + o, A::ldcg(nb + o));  // frozen: carry z to the next step
                continue;
            }
            if constexpr (kFix) {
                if (fixp) {  // s == SB: the halves P (with x) and Q (with z) in fixed point
                    double u[SB + 1], po[SB], qo[SB], v[SB], pq[SB];
#pragma unroll
                    for (int c = 0; c <= SB; c++) u[c] = __ldcg(nb + c * nR + o);
#pragma unroll
                    for (int l = 0; l < SB; l++) {
                        po[l] = __ldcg(ob + l * nR + o);
                        qo[l] = __ldcg(ob + (SB + 1 + l) * nR + o);
                    }
                    double x = __ldcg(xw + o), za = 0.0;
#pragma unroll
                    for (int j = 0; j < SB; j++) v[j] = u[j];
                    if (!fix_update_group<SB>(v, po, s_cf[r], s_fc[r], s_rng[r][0], s_rng[r][1], pq))
                        fma_update_group<SB>(v, po, &s_beta[r][0], pq);
#pragma unroll
                    for (int j = 0; j < SB; j++) {
                        __stcs(nb + j * nR + o, pq[j]);
                        x = ::fma(pq[j], s_alpha[r][j], x);
                    }
#pragma unroll
                    for (int j = 0; j < SB; j++) v[j] = u[j + 1];
                    if (!fix_update_group<SB>(v, qo, s_cf[r], s_fc[r], s_rng[r][0], s_rng[r][1], pq))
                        fma_update_group<SB>(v, qo, &s_beta[r][0], pq);
#pragma unroll
                    for (int j = 0; j < SB; j++) {
                        __stcs(nb + (SB + 1 + j) * nR + o, pq[j]);
                        za = ::fma(pq[j], s_alpha[r][j], za);
                    }
                    const double z = u[0] - za;
                    xw[o] = x;
                    ob[o] = z;
                    const double rn = (yb.diag ? __ldg(reinterpret_cast<const double*>(yb.diag) + i) : yb.diag_c) * z;
                    rr = ::fma(rn, rn, rr);
                    rz = ::fma(rn, z, rz);
                    continue;
                }
            }
            Rv u[SB + 1], po[SB], qo[SB];
#pragma unroll
            for (int c = 0; c <= SB; c++)
                if (c <= s) u[c] = A::ldcg(nb + c * nR + o);
            if (kk > 0) {
#pragma unroll
                for (int l = 0; l < SB; l++)
                    if (l < s) {
                        po[l] = A::ldcg(ob + l * nR + o);
                        qo[l] = A::ldcg(ob + (s + 1 + l) * nR + o);
                    }
            }
            Rv x = A::ldcg(xw + o), za = A::zero();
#pragma unroll
            for (int jj = 0; jj < SB; jj++) {
                if (jj >= s) continue;
                Rv p = u[jj], q = u[jj + 1];
                if (kk > 0) {
#pragma unroll
                    for (int l = 0; l < SB; l++)
                        if (l < s) {
                            const Rv bl = s_beta[r][l + jj * s];
                            p = A::fma(po[l], bl, p);
                            q = A::fma(qo[l], bl, q);
                        }
                    A::st_stream(nb + jj * nR + o, p);
                }
                A::st_stream(nb + (s + 1 + jj) * nR + o, q);
                const Rv al = s_alpha[r][jj];
                x = A::fma(p, al, x);
                za = A::fma(q, al, za);
            }
            const Rv z = A::sub(u[0], za);
            A::st(xw + o, x);
            A::st(ob + o, z);
            const Rv rn = A::mul(yb.diag ? A::ldg(reinterpret_cast<const S*>(yb.diag) + i) : dcst, z);
            rr = A::fma(rn, rn, rr);
            rz = A::fma(rn, z, rz);
        }
        double out = 0.0;
        cta_sum_slots<A>(rr, slot, R, red, &out);
        if (threadIdx.x < R) y.upart[(size_t)threadIdx.x * y.items + li] = out;
        cta_sum_slots<A>(rz, slot, R, red, &out);
        if (threadIdx.x < R) y.upart[(size_t)(R + threadIdx.x) * y.items + li] = out;
    }
}

#undef ITEM_MAP

// The whole batched solve in one cooperative launch: the phases separated by
// grid-wide barriers (bounded waits).
template <class A, int SB>
__global__ void __launch_bounds__(kBThreads, 3) k_batch(BArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.g->t0 = globaltimer();
    ph_init<A>(a, blockIdx.x, gridDim.x);
    if (!grid_sync(a.g, a.skip_cta, a.wait_ns)) return;
    for (;;) {
        for (int j = 0; j < a.s; j++) {
            ph_level<A, false>(a, j, blockIdx.x, gridDim.x);
            if (!grid_sync(a.g, a.skip_cta, a.wait_ns)) return;
        }
        ph_solve<A>(a, blockIdx.x, gridDim.x);
        if (!grid_sync(a.g, a.skip_cta, a.wait_ns)) return;
        if (*(volatile int*)&a.g->finished >= a.nsys) break;
        ph_update<A, SB>(a, blockIdx.x, gridDim.x);
        if (!grid_sync(a.g, a.skip_cta, a.wait_ns)) return;
    }
}

// One launch per phase (captured in a CUDA graph per outer step).  Launches
// queued after every system finished return at once.
__device__ __forceinline__ bool batch_done(const BArgs& a) { return *(volatile int*)&a.g->finished >= a.nsys; }

template <class A>
__global__ void __launch_bounds__(kBThreads) k_bp_init(BArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.g->t0 = globaltimer();
    ph_init<A>(a, blockIdx.x, gridDim.x);
}

template <class A, int KIND>
__global__ void __launch_bounds__(kBThreads) k_bp_level(BArgs a, int j) {
    if (batch_done(a)) return;
    ph_level<A, true, KIND>(a, j, blockIdx.x, gridDim.x);
}

// Kind 3 (FP64 27-point Laplacian-class systems), built for 2 CTAs per SM.
template <class A>
__global__ void __launch_bounds__(kBThreads, 2) k_bp_level27(BArgs a, int j) {
    if (batch_done(a)) return;
    ph_level<A, true, 3>(a, j, blockIdx.x, gridDim.x);
}

template <class A>
__global__ void __launch_bounds__(kBThreads) k_bp_solve(BArgs a) {
    if (batch_done(a)) return;
    ph_solve<A>(a, blockIdx.x, gridDim.x);
}

template <class A, int SB>
__global__ void __launch_bounds__(kBThreads, 3) k_bp_update(BArgs a) {
    if (batch_done(a)) return;
    ph_update<A, SB>(a, blockIdx.x, gridDim.x);
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
    int persistent;              // one cooperative launch instead of per-phase launches
    int fma_update;              // SSCG_FMA_UPDATE
    int g_init, g_level, g_level_dia, g_level_dia27, g_update;  // per-phase grids (CSR, diagonal-form,
                                                                 // FP64 27-point diagonal-form levels)
    int has_csr, has_dia, has_dia27;                            // which level kernels an outer step launches
    cudaGraphExec_t step_exec;   // per-phase mode: one outer step
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
    int64_t last_launches;       // kernels the last solve ran (graph nodes included)
    int fault_cta = -1;          // armed barrier fault for the next solve (sscg_batch_inject_barrier_fault)
    unsigned long long fault_wait_ns = 0;
};

namespace {

struct BLayout {
    size_t bytes;
    std::vector<size_t> off_blk0, off_blk1, off_xw, off_l, off_u;
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
        L.off_blk0.push_back(take((2 * (size_t)s + 1) * nR * eb));
        L.off_blk1.push_back(take((2 * (size_t)s + 1) * nR * eb));
        L.off_xw.push_back(take(nR * eb));
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
    if (o->arith == SSCG_ARITH_DF64 && o->s > kMaxSDf64Monomial)
        return set_err(ctx, SSCG_ERR_INVALID, "double-float arithmetic takes the monomial basis up to s = %d; use f64",
                       kMaxSDf64Monomial);
    if (o->maxit < 0 || !(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad maxit or tol");
    for (int k = 0; k < nsys; k++) {
        if (!mats[k]) return set_err(ctx, SSCG_ERR_INVALID, "system %d: null matrix", k);
        if (o->arith != SSCG_ARITH_F64 && mats[k]->out_of_f32)
            return set_err(ctx, SSCG_ERR_INVALID, "system %d: values outside FP32's normal range; use f64", k);
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

BArgs make_args(const sscg_batch* b, int tuning, int maxit) {
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
    a.skip_cta = b->fault_cta;
    a.wait_ns = b->fault_cta >= 0 ? b->fault_wait_ns : kBarrierTimeoutNs;
    a.fma_update = b->fma_update;
    return a;
}

template <class A, int SB>
int launch_persistent(sscg_batch* b, int tuning, int maxit, cudaStream_t st) {
    const BArgs a = make_args(b, tuning, maxit);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(kBThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    SSCG_CUDA(b->ctx, cudaLaunchKernelEx(&cfg, k_batch<A, SB>, a));
    return SSCG_OK;
}

// Per-phase mode: the init launch, and the launches of one outer step.
template <class A, int SB>
int launch_init(sscg_batch* b, int tuning, int maxit, cudaStream_t st) {
    const BArgs a = make_args(b, tuning, maxit);
    k_bp_init<A><<<b->g_init, kBThreads, 0, st>>>(a);
    SSCG_CUDA(b->ctx, cudaGetLastError());
    return SSCG_OK;
}

template <class A, int SB>
int launch_step(sscg_batch* b, int tuning, int maxit, cudaStream_t st) {
    const BArgs a = make_args(b, tuning, maxit);
    for (int j = 0; j < b->s; j++) {
        if (b->has_csr) k_bp_level<A, 1><<<b->g_level, kBThreads, kLevelSmem, st>>>(a, j);
        if (b->has_dia) k_bp_level<A, 2><<<b->g_level_dia, kBThreads, kLevelSmem, st>>>(a, j);
        if (b->has_dia27) k_bp_level27<A><<<b->g_level_dia27, kBThreads, kLevelSmem, st>>>(a, j);
    }
    k_bp_solve<A><<<std::min(b->nsys, kMaxGrid), kBThreads, 0, st>>>(a);
    k_bp_update<A, SB><<<b->g_update, kBThreads, 0, st>>>(a);
    SSCG_CUDA(b->ctx, cudaGetLastError());
    return SSCG_OK;
}

enum LaunchKind { L_PERSISTENT = 0, L_INIT = 1, L_STEP = 2 };

template <class A, int SB>
int launch_kind(sscg_batch* b, int kind, int tuning, int maxit, cudaStream_t st) {
    if (kind == L_PERSISTENT) return launch_persistent<A, SB>(b, tuning, maxit, st);
    if (kind == L_INIT) return launch_init<A, SB>(b, tuning, maxit, st);
    return launch_step<A, SB>(b, tuning, maxit, st);
}

// Launch on `st` (default: the context's stream).
int launch_any(sscg_batch* b, int kind, int tuning, int maxit, cudaStream_t st) {
    if (b->arith == SSCG_ARITH_F64)
        return b->s <= 4 ? launch_kind<ArithF64, 4>(b, kind, tuning, maxit, st)
                         : launch_kind<ArithF64, kMaxSB>(b, kind, tuning, maxit, st);
    return b->s <= 4 ? launch_kind<ArithDF64, 4>(b, kind, tuning, maxit, st)
                     : launch_kind<ArithDF64, kMaxSB>(b, kind, tuning, maxit, st);
}

int launch_any(sscg_batch* b, int kind, int tuning, int maxit) {
    return launch_any(b, kind, tuning, maxit, b->ctx->stream);
}

template <class A, int SB>
int phase_grids(sscg_batch* b) {
    sscg_ctx* ctx = b->ctx;
    auto grid_of = [&](auto kernel) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBThreads, 0) != cudaSuccess || per < 1) per = 1;
        return std::min(kMaxGrid, ctx->sm_count * std::min(per, 8));
    };
    b->g_init = grid_of(k_bp_init<A>);
    auto level_grid = [&](auto kernel) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLevelSmem);
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBThreads, kLevelSmem) != cudaSuccess || per < 1)
            per = 1;
        return std::min(kMaxGrid, ctx->sm_count * std::min(per, 8));
    };
    b->g_level = level_grid(k_bp_level<A, 1>);
    b->g_level_dia = level_grid(k_bp_level<A, 2>);
    b->g_level_dia27 = level_grid(k_bp_level27<A>);
    b->g_update = grid_of(k_bp_update<A, SB>);
    int per = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch<A, SB>, kBThreads, 0);
    if (e != cudaSuccess || per < 1)
        return set_err(ctx, SSCG_ERR_CUDA, "batched kernel cannot be resident: %s", cudaGetErrorString(e));
    b->grid = per * ctx->sm_count;  // co-resident grid of the cooperative kernel
    cudaGetLastError();
    return SSCG_OK;
}

int setup_grids(sscg_batch* b) {
    if (b->arith == SSCG_ARITH_F64) return b->s <= 4 ? phase_grids<ArithF64, 4>(b) : phase_grids<ArithF64, kMaxSB>(b);
    return b->s <= 4 ? phase_grids<ArithDF64, 4>(b) : phase_grids<ArithDF64, kMaxSB>(b);
}

// Reset the per-solve state on the stream: control blocks zeroed.
int reset_state(sscg_batch* b) {
    sscg_ctx* ctx = b->ctx;
    SSCG_CUDA(ctx, cudaMemsetAsync(b->d_g, 0, sizeof(GCtl), ctx->stream));
    SSCG_CUDA(ctx, cudaMemsetAsync(b->d_bctl, 0, sizeof(BCtl) * b->nsys, ctx->stream));
    SSCG_CUDA(ctx, cudaMemsetAsync(b->d_rc, 0, sizeof(Ctrl) * b->total_rhs, ctx->stream));
    return SSCG_OK;
}

// One solve without a graph or polling: the cooperative launch, or the init
// launch and maxit + 3 outer-step launches (each returns at once after the
// last system finished).  Used by the autotuner and when capture fails.
int run_plain(sscg_batch* b, int tuning, int maxit) {
    if (b->persistent) return launch_any(b, L_PERSISTENT, tuning, maxit);
    if (int rc = launch_any(b, L_INIT, tuning, maxit)) return rc;
    for (int q = 0; q < maxit + 3; q++)
        if (int rc = launch_any(b, L_STEP, tuning, maxit)) return rc;
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
                if ((rc = run_plain(b, 1, 2))) break;
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

// Capture the graph a solve replays: the whole solve for the cooperative mode
// (state reset, pointer upload, kernel, results back), one outer step
// (s level launches, the solve launch, the update launch) for the per-phase
// mode.  On a capture failure the plan launches directly.
void build_graph(sscg_batch* b) {
    // capture on a private stream: the context's stream may be the legacy
    // default stream, which cannot be captured; the graph is replayed on it
    cudaStream_t st = nullptr;
    cudaGraph_t graph = nullptr;
    b->graph_ok = 0;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(st);
        return;
    }
    bool ok = true;
    if (b->persistent) {
        ok = cudaMemsetAsync(b->d_g, 0, sizeof(GCtl), st) == cudaSuccess &&
             cudaMemsetAsync(b->d_bctl, 0, sizeof(BCtl) * b->nsys, st) == cudaSuccess &&
             cudaMemsetAsync(b->d_rc, 0, sizeof(Ctrl) * b->total_rhs, st) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(b->d_io, b->h_io, sizeof(double*) * 2 * b->nsys, cudaMemcpyHostToDevice, st) ==
                       cudaSuccess;
        ok = ok && launch_any(b, L_PERSISTENT, 0, b->maxit, st) == SSCG_OK;
        ok = ok && cudaMemcpyAsync(b->h_rc, b->d_rc, sizeof(Ctrl) * b->total_rhs, cudaMemcpyDeviceToHost, st) ==
                       cudaSuccess;
        ok = ok && cudaMemcpyAsync(b->h_bctl, b->d_bctl, sizeof(BCtl) * b->nsys, cudaMemcpyDeviceToHost, st) ==
                       cudaSuccess;
        ok = ok && cudaMemcpyAsync(b->h_g, b->d_g, sizeof(GCtl), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    } else {
        ok = launch_any(b, L_STEP, 0, b->maxit, st) == SSCG_OK;
    }
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (ok && e == cudaSuccess && graph) {
        cudaGraphExec_t ex = nullptr;
        if (cudaGraphInstantiate(&ex, graph, 0) == cudaSuccess) {
            b->graph_ok = 1;
            if (b->persistent) b->exec = ex;
            else b->step_exec = ex;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(st);
    cudaGetLastError();
}

// Per-phase mode: init launch, then outer steps replayed in chunks until the
// device's count of finished systems reaches nsys (read back through pinned
// memory one chunk behind, so the host never stalls the stream).
int run_phases(sscg_batch* b) {
    sscg_ctx* ctx = b->ctx;
    cudaStream_t st = ctx->stream;
    if (int rc = reset_state(b)) return rc;
    SSCG_CUDA(ctx, cudaMemcpyAsync(b->d_io, b->h_io, sizeof(double*) * 2 * b->nsys, cudaMemcpyHostToDevice, st));
    if (int rc = launch_any(b, L_INIT, 0, b->maxit)) return rc;
    b->last_launches = 1;
    const int limit = b->maxit + 4, per_chunk = 8;
    ChunkPoll poll;
    SSCG_CUDA(ctx, poll.init());
    int launched = 0, rc = SSCG_OK;
    while (launched < limit) {
        const int c = std::min(per_chunk, limit - launched);
        for (int q = 0; q < c && rc == SSCG_OK; q++) {
            if (b->graph_ok) {
                if (cudaGraphLaunch(b->step_exec, st) != cudaSuccess)
                    rc = set_err(ctx, SSCG_ERR_CUDA, "graph launch: %s", cudaGetErrorString(cudaGetLastError()));
            } else {
                rc = launch_any(b, L_STEP, 0, b->maxit);
            }
        }
        if (rc) break;
        launched += c;
        b->last_launches += (int64_t)c * (b->s * (b->has_csr + b->has_dia + b->has_dia27) + 2);  // levels, solves, update
        int fin = 0;
        cudaError_t pe = cudaSuccess;
        const bool got = poll.step(ctx->pinned, &b->d_g->finished, st, &fin, &pe);
        if (pe != cudaSuccess) {
            rc = set_err(ctx, SSCG_ERR_CUDA, "polling: %s", cudaGetErrorString(pe));
            break;
        }
        if (got && fin >= b->nsys) break;
    }
    if (rc) return rc;
    SSCG_CUDA(ctx, cudaMemcpyAsync(b->h_rc, b->d_rc, sizeof(Ctrl) * b->total_rhs, cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaMemcpyAsync(b->h_bctl, b->d_bctl, sizeof(BCtl) * b->nsys, cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaMemcpyAsync(b->h_g, b->d_g, sizeof(GCtl), cudaMemcpyDeviceToHost, st));
    return SSCG_OK;
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
        const bool f64 = opts->arith == SSCG_ARITH_F64;
        if (m->dia) {
            // constant-coefficient diagonal form: masks, offsets, values; D is one constant
            if (f64 && m->dia_k == 27 && m->dia_lap && m->dia_cen == 13) b->has_dia27 = 1;
            else b->has_dia = 1;
            y.dmask = m->dia_mask;
            y.dk = m->dia_k;
            y.dcen = m->dia_cen;
            y.dlap = m->dia_lap;
            y.dco = (float)m->dia_co;
            for (int t = 0; t < m->dia_k; t++) {
                y.doff[t] = m->dia_off[t];
                y.dcf[t] = (float)m->dia_c[t];
            }
            y.dinv = nullptr;
            y.diag = nullptr;
            y.dinv_c = m->dia_dinv;
            y.diag_c = m->dia_d;
        } else {
            b->has_csr = 1;
            y.dinv = f64 ? (const void*)m->dinv : (const void*)m->dinv_df;
            y.diag = f64 ? (const void*)m->diag : (const void*)m->diag_df;
        }
        y.blk[0] = base + L.off_blk0[k];
        y.blk[1] = base + L.off_blk1[k];
        y.xw = base + L.off_xw[k];
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
    b->persistent = (opts->flags & SSCG_BATCH_PERSISTENT) ? 1 : 0;
    b->fma_update = (opts->flags & SSCG_FMA_UPDATE) ? 1 : 0;
    if (int rc = setup_grids(b)) return fail(rc);
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
    if (b->step_exec) cudaGraphExecDestroy(b->step_exec);
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
    b->last_launches = 1;  // the persistent mode: one cooperative kernel
    const bool fault = b->fault_cta >= 0;  // an armed fault runs outside the captured graph
    if (!b->persistent) {
        if (int rc = run_phases(b)) return rc;
    } else if (b->graph_ok && !fault) {
        SSCG_CUDA(ctx, cudaGraphLaunch(b->exec, st));
    } else {
        if (int rc = reset_state(b)) return rc;
        SSCG_CUDA(ctx, cudaMemcpyAsync(b->d_io, b->h_io, sizeof(double*) * 2 * b->nsys, cudaMemcpyHostToDevice, st));
        const int lrc = launch_any(b, L_PERSISTENT, 0, b->maxit);
        b->fault_cta = -1;  // disarmed after one solve
        if (lrc) return lrc;
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

int sscg_batch_inject_barrier_fault(sscg_batch* b, int cta, int wait_ms) {
    if (!b) return SSCG_ERR_INVALID;
    if (cta == -1) {
        b->fault_cta = -1;
        return SSCG_OK;
    }
    if (!b->persistent) return set_err(b->ctx, SSCG_ERR_INVALID, "barrier faults need a persistent plan");
    if (cta < 0 || cta >= b->grid) return set_err(b->ctx, SSCG_ERR_INVALID, "CTA %d outside the grid of %d", cta, b->grid);
    if (wait_ms < 1 || wait_ms > 10000) return set_err(b->ctx, SSCG_ERR_INVALID, "wait_ms must lie in 1..10000");
    b->fault_cta = cta;
    b->fault_wait_ns = (unsigned long long)wait_ms * 1000000ull;
    return SSCG_OK;
}

int sscg_batch_props(const sscg_batch* b, int* tile_rows, int* grid, int* graph, float* last_ms) {
    if (!b) return SSCG_ERR_INVALID;
    if (tile_rows)
        for (int k = 0; k < b->nsys; k++) tile_rows[k] = b->T[k];
    if (grid) *grid = b->persistent ? b->grid : b->g_update;
    if (graph) *graph = b->graph_ok;
    if (last_ms) *last_ms = b->last_ms;
    return SSCG_OK;
}

int sscg_batch_launches(const sscg_batch* b, int64_t* launches) {
    if (!b || !launches) return SSCG_ERR_INVALID;
    *launches = b->last_launches;
    return SSCG_OK;
}

}  // extern "C"
