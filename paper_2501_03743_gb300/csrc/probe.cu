// Arithmetic throughput probes (include/sscg_probe.h): one kernel per
// instruction kind, every thread running kChains independent dependency
// chains so that latency is hidden, over a full-device grid, timed with CUDA
// events.  Results are kept alive through a comparison against a value the
// chains never reach, so no store happens and the compiler cannot drop the
// work.
#include "../../include/sscg_probe.h"
#include "internal.h"
#include "small.cuh"

namespace {

constexpr int kChains = 8;    // independent chains per thread (FP64, FP32, integer kinds)
constexpr int kMmaAcc = 8;    // independent 8x8 accumulators per warp (DMMA kind)
constexpr int kProbeThreads = 256;

__device__ double g_probe_sink;  // written only if a chain hits an impossible value

__device__ __forceinline__ void dmma_m8n8k4(double& d0, double& d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ double dfma_chains(long long iters, double seed, double m, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed + k;
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fma(a[k], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) t += a[k];
    return t;
}

__device__ __forceinline__ double dmma_chains(long long iters, double seed) {
    double acc[kMmaAcc][2];
#pragma unroll
    for (int k = 0; k < kMmaAcc; k++) acc[k][0] = acc[k][1] = seed;
    const double a = 1e-3 + 1e-6 * (threadIdx.x & 31), b = 1e-3 - 1e-6 * (threadIdx.x & 31);
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kMmaAcc; k++) dmma_m8n8k4(acc[k][0], acc[k][1], a, b);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kMmaAcc; k++) t += acc[k][0] + acc[k][1];
    return t;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe(long long iters_a, long long iters_b, double seed) {
    double t = 0.0;
    if constexpr (KIND == SSCG_PROBE_DFMA) {
        t = dfma_chains(iters_a, seed, 1.0 - 0x1p-30, 1e-7);
    } else if constexpr (KIND == SSCG_PROBE_DADD) {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = seed + k;
        const double c = 1e-9 * seed;
        for (long long it = 0; it < iters_a; it++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = a[k] + c;
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k];
    } else if constexpr (KIND == SSCG_PROBE_DMUL) {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = seed + k;
        const double m = 1.0 - 0x1p-30 * seed;
        for (long long it = 0; it < iters_a; it++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = a[k] * m;
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k];
    } else if constexpr (KIND == SSCG_PROBE_DMMA) {
        t = dmma_chains(iters_a, seed);
    } else if constexpr (KIND == SSCG_PROBE_DFMA_DMMA) {
        // warp-uniform split: even warps on the FP64 FMA pipe, odd warps on the tensor instruction
        if (((threadIdx.x >> 5) & 1) == 0) t = dfma_chains(iters_a, seed, 1.0 - 0x1p-30, 1e-7);
        else t = dmma_chains(iters_b, seed);
    } else if constexpr (KIND == SSCG_PROBE_FFMA) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = (float)seed + k;
        const float m = 1.0f - 0x1p-20f, c = 1e-6f;
#pragma unroll 4
        for (long long it = 0; it < iters_a; it++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) t += a[k];
    } else if constexpr (KIND == SSCG_PROBE_IALU) {
        unsigned x[kChains];
        const unsigned y = 0x9E3779B9u ^ (unsigned)seed, z = 0x7F4A7C15u + threadIdx.x;
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = threadIdx.x * 2654435761u + k;
        // each step mixes a neighbouring chain in, so the chains cannot be run one after another
#pragma unroll 4
        for (long long it = 0; it < iters_a; it++) {
            unsigned nx[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) nx[k] = (x[k] ^ x[(k + 1) % kChains] ^ y) + z;
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = nx[k];
        }
        unsigned u = 0;
#pragma unroll
        for (int k = 0; k < kChains; k++) u ^= x[k];
        t = (double)u - 1.0;  // -1 only if every chain ends at 0
    } else if constexpr (KIND == SSCG_PROBE_IMAD_WIDE) {
        // the low word of each 64-bit sum is the next multiplicand (a register, no instruction)
        long long c[kChains];
        const int m = (int)(2654435761u ^ (unsigned)seed);
#pragma unroll
        for (int k = 0; k < kChains; k++) c[k] = (long long)threadIdx.x * 40503 + k;
#pragma unroll 4
        for (long long it = 0; it < iters_a; it++) {
            long long nc[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) {
                const int a = (int)c[k];
                asm volatile("mad.wide.s32 %0, %1, %2, %3;" : "=l"(nc[k]) : "r"(a), "r"(m), "l"(c[(k + 1) % kChains]));
            }
#pragma unroll
            for (int k = 0; k < kChains; k++) c[k] = nc[k];
        }
        long long u = 0;
#pragma unroll
        for (int k = 0; k < kChains; k++) u ^= c[k];
        t = (double)(u & 0xFFFF) - 1.0;  // -1 only if every chain's low bits end at 0
    } else if constexpr (KIND == SSCG_PROBE_I2F64) {
        // the bit pattern of each converted value is the next integer (a register, no instruction)
        double d[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) d[k] = seed + k;
#pragma unroll 4
        for (long long it = 0; it < iters_a; it++) {
            double nd[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) {
                const long long v = __double_as_longlong(d[(k + 1) % kChains]);
                asm volatile("cvt.rn.f64.s64 %0, %1;" : "=d"(nd[k]) : "l"(v));
            }
#pragma unroll
            for (int k = 0; k < kChains; k++) d[k] = nd[k];
        }
#pragma unroll
        for (int k = 0; k < kChains; k++) t += d[k];
    } else if constexpr (KIND == SSCG_PROBE_F2I64) {
        // the converted integer with the exponent of 2^52 set is the next FP64 value (one LOP3 on
        // its high word): every value lies in [2^52, 2^53)
        long long v[kChains];
#pragma unroll
        for (int k = 0; k < kChains; k++) v[k] = (long long)(seed * 1e15) + k;
#pragma unroll 4
        for (long long it = 0; it < iters_a; it++) {
            long long nv[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) {
                const double d = __longlong_as_double(v[(k + 1) % kChains] | 0x4330000000000000ll);
                asm volatile("cvt.rzi.s64.f64 %0, %1;" : "=l"(nv[k]) : "d"(d));
            }
#pragma unroll
            for (int k = 0; k < kChains; k++) v[k] = nv[k];
        }
        long long u = 0;
#pragma unroll
        for (int k = 0; k < kChains; k++) u ^= v[k];
        t = (double)(u & 0xFFFF) - 1.0;
    } else {
        unsigned x[kChains];
        const unsigned m = 2654435761u ^ (unsigned)seed;
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = threadIdx.x + k;
#pragma unroll 4
        for (long long it = 0; it < iters_a; it++) {
            unsigned nx[kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) nx[k] = x[k] * m + x[(k + 1) % kChains];
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = nx[k];
        }
        unsigned u = 0;
#pragma unroll
        for (int k = 0; k < kChains; k++) u ^= x[k];
        t = (double)u - 1.0;  // -1 only if every chain ends at 0
    }
    if (t == -1.0) g_probe_sink = t;  // never true: keeps the chains live
}

template <int KIND>
int run_probe(sscg_ctx* ctx, long long ia, long long ib, double* ops, double* ms) {
    int per_sm = 0;
    SSCG_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe<KIND>, kProbeThreads, 0));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    const long long grid = (long long)ctx->sm_count * per_sm;
    cudaEvent_t e0, e1;
    SSCG_CUDA(ctx, cudaEventCreate(&e0));
    SSCG_CUDA(ctx, cudaEventCreate(&e1));
    SSCG_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
    k_probe<KIND><<<(unsigned)grid, kProbeThreads, 0, ctx->stream>>>(ia, ib, 1.0 + 1e-3 * KIND);
    cudaError_t le = cudaGetLastError();
    SSCG_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
    SSCG_CUDA(ctx, cudaEventSynchronize(e1));
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (le != cudaSuccess) return sscg::set_err(ctx, SSCG_ERR_CUDA, "probe launch: %s", cudaGetErrorString(le));
    const double threads = (double)grid * kProbeThreads, warps = threads / 32.0;
    double n = 0.0;
    switch (KIND) {
        case SSCG_PROBE_DMMA: n = warps * (double)ia * kMmaAcc * 256.0; break;
        case SSCG_PROBE_DFMA_DMMA:
            n = threads / 2 * (double)ia * kChains + warps / 2 * (double)ib * kMmaAcc * 256.0;
            break;
        case SSCG_PROBE_IALU: n = threads * (double)ia * kChains * 2.0; break;
        default: n = threads * (double)ia * kChains;
    }
    *ms = t;
    *ops = t > 0.f ? n / (t * 1e-3) : 0.0;
    return SSCG_OK;
}

}  // namespace

extern "C" int sscg_probe_rate(sscg_ctx* ctx, int kind, int64_t iters_a, int64_t iters_b, double* ops_per_s,
                               double* ms) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (!ops_per_s || !ms) return sscg::set_err(ctx, SSCG_ERR_INVALID, "null output");
    const int64_t lim = (int64_t)1 << 40;
    if (iters_a <= 0 || iters_a > lim || (kind == SSCG_PROBE_DFMA_DMMA && (iters_b <= 0 || iters_b > lim)))
        return sscg::set_err(ctx, SSCG_ERR_INVALID, "iteration counts must lie in 1..2^40");
    switch (kind) {
        case SSCG_PROBE_DFMA: return run_probe<SSCG_PROBE_DFMA>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_DADD: return run_probe<SSCG_PROBE_DADD>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_DMUL: return run_probe<SSCG_PROBE_DMUL>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_DMMA: return run_probe<SSCG_PROBE_DMMA>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_DFMA_DMMA: return run_probe<SSCG_PROBE_DFMA_DMMA>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_FFMA: return run_probe<SSCG_PROBE_FFMA>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_IALU: return run_probe<SSCG_PROBE_IALU>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_IMAD: return run_probe<SSCG_PROBE_IMAD>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_IMAD_WIDE: return run_probe<SSCG_PROBE_IMAD_WIDE>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_I2F64: return run_probe<SSCG_PROBE_I2F64>(ctx, iters_a, iters_b, ops_per_s, ms);
        case SSCG_PROBE_F2I64: return run_probe<SSCG_PROBE_F2I64>(ctx, iters_a, iters_b, ops_per_s, ms);
        default: return sscg::set_err(ctx, SSCG_ERR_INVALID, "unknown probe kind %d", kind);
    }
}

namespace {

using sscg::Ctrl;
using sscg::SmallScratch;

__device__ Ctrl g_probe_ctrl;               // moments for the monomial step
__device__ long long g_probe_cycles[5];     // sums of cycles; [4]: failed factorisations

// One warp: the small-solve routines on fixed inputs, timed with clock64.
__global__ void __launch_bounds__(32) k_probe_small(int s, int reps) {
    __shared__ SmallScratch sc;
    __shared__ double A0[64], L[64], X[64], b[8], rv[8];
    const int lane = threadIdx.x;
    // A0 = diag(2 + i) + 0.1 (all ones): SPD
    for (int e = lane; e < s * s; e += 32) A0[e] = (e % s == e / s ? 2.0 + e % s : 0.0) + 0.1;
    // mu_k = sum_m w_m lam_m^k over 16 points lam_m in (0, 2): Hankel matrices SPD for s <= 8
    if (lane < 2 * s) {
        double mu = 0.0;
        for (int m = 0; m < 16; m++) {
            const double lam = 0.0625 + 0.118 * m, w = 1.0 + 0.05 * m;
            double p = w;
            for (int q = 0; q < lane; q++) p *= lam;
            mu += p;
        }
        g_probe_ctrl.mu[lane] = mu;
    }
    __syncwarp();
    long long c[4] = {0, 0, 0, 0};
    long long fails = 0;
    for (int r = 0; r < reps; r++) {
        for (int e = lane; e < s * s; e += 32) {
            L[e] = A0[e];
            X[e] = e % s == e / s ? 1.0 : 0.0;
        }
        if (lane < s) b[lane] = 1.0 + lane;
        __syncwarp();
        const long long t0 = clock64();
        bool ok = sscg::warp_cholesky(L, s, rv);
        const long long t1 = clock64();
        ok = sscg::warp_chol_solve(L, s, b, 1, rv) && ok;
        const long long t2 = clock64();
        ok = sscg::warp_chol_solve(L, s, X, s, rv) && ok;
        const long long t3 = clock64();
        const int st = sscg::warp_sw_monomial(&g_probe_ctrl, s, 0, &sc);
        const long long t4 = clock64();
        c[0] += t1 - t0;
        c[1] += t2 - t1;
        c[2] += t3 - t2;
        c[3] += t4 - t3;
        if (!ok || st != 0) fails++;
    }
    if (lane == 0) {
        for (int k = 0; k < 4; k++) g_probe_cycles[k] = c[k];
        g_probe_cycles[4] = fails;
    }
}

}  // namespace

extern "C" int sscg_probe_small_solve(sscg_ctx* ctx, int s, int reps, double* cycles) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (!cycles) return sscg::set_err(ctx, SSCG_ERR_INVALID, "null output");
    if (s < 1 || s > 8 || reps < 1 || reps > 100000)
        return sscg::set_err(ctx, SSCG_ERR_INVALID, "s must lie in 1..8 and reps in 1..100000");
    k_probe_small<<<1, 32, 0, ctx->stream>>>(s, reps);
    SSCG_CUDA(ctx, cudaGetLastError());
    long long h[5];
    SSCG_CUDA(ctx, cudaMemcpyFromSymbolAsync(h, g_probe_cycles, sizeof(h), 0, cudaMemcpyDeviceToHost, ctx->stream));
    SSCG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h[4] != 0) return sscg::set_err(ctx, SSCG_BREAKDOWN, "a probe factorisation failed");
    for (int k = 0; k < 4; k++) cycles[k] = (double)h[k] / reps;
    return SSCG_OK;
}
