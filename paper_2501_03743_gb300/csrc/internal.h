// Host-side definitions shared by the translation units of libsscg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>

#include "../../include/sscg.h"

struct sscg_ctx {
    cudaStream_t stream;
    int device;
    int sm_count;
    char err[512];
    volatile int* pinned;  // small page-locked host buffer for polling reads (8 slots)
    cudaEvent_t* ev;       // event pool for SSCG_PROFILE
    int ev_cap;
};

struct sscg_mat {
    int64_t n, nnz;
    // device arrays inside the caller's storage
    int32_t* rowptr;
    int32_t* col;
    double* val;     // FP64 values
    float* vhi;      // FP32 part of every value (exact when values_exact_fp32)
    float* vlo;      // FP32 remainder val - vhi
    double* diag;
    double* dinv;    // 1 / diag
    float2* dinv_df; // 1 / diag as a double-float
    float2* diag_df; // diag as a double-float
    float* dinv_f;   // 1 / diag rounded to FP32 (mixed-precision basis)
    // properties
    int64_t bandwidth;
    int exact_fp32;
    int out_of_f32;  // some nonzero value lies outside FP32's normal range: df64 / mixed solves refuse
    int max_row_nnz;
    int max_tile_nnz;  // largest nnz count of a 256-row tile
    double dmin, dmax;
    // preconditioner
    int prec, degree;
    double plmin, plmax;
    // spectral-bound network for automatic Chebyshev-basis intervals
    // (device blob owned by the caller), or null
    const double* bounds_model;
    int bounds_h;
    // constant-coefficient diagonal form (dia != 0): every row's entries lie
    // on dia_k fixed offsets, each offset carrying one FP32-exact value;
    // dia_mask[i] bit t set when row i holds offset t
    int dia, dia_k;
    int dia_off[32];
    double dia_c[32];
    uint32_t* dia_mask;
    double dia_d, dia_dinv;  // the diagonal's value and its inverse
    int dia_cen;             // index of offset 0 among the sorted offsets
    int dia_lap;             // every off-centre value equals dia_co
    double dia_co;
    int64_t dia_reach;       // max |offset|
};

namespace sscg {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-provided region.
struct Carve {
    char* base;
    size_t cap, used;
    Carve(void* b, size_t c) : base((char*)b), cap(c), used(0) {}
    template <class T>
    T* take(size_t count) {
        size_t off = align_up(used, 256);
        used = off + align_up(count * sizeof(T), 256);
        return base ? (T*)(base + off) : nullptr;
    }
    bool ok() const { return used <= cap; }
};

// Margin (elements) carved before and after every vector that a
// diagonal-form level gathers from, so its paired-row gathers need no clamps
// (spmv_dia_df); 0 for a CSR matrix.
inline size_t dia_margin(const sscg_mat* m) {
    return m->dia ? align_up((size_t)m->dia_reach + 2, 32) : 0;
}

// Which diagonal-form SpMV a double-float kernel is built with: 0 CSR; 1
// clamped (vectors without margins); 7 / 27 the Laplacian class (all
// off-centre values equal, offset 0 in the middle) with that many offsets;
// 2 any other diagonal form over margined vectors.
inline int dia_mode(const sscg_mat* m, bool margins) {
    if (!m->dia) return 0;
    if (!margins) return 1;
    if (m->dia_lap && m->dia_k == 7 && m->dia_cen == 3) return 7;
    if (m->dia_lap && m->dia_k == 27 && m->dia_cen == 13) return 27;
    return 2;
}

inline int set_err(sscg_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define SSCG_CUDA(ctx, call)                                                                   \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ::sscg::set_err((ctx), SSCG_ERR_CUDA, "%s: %s (%s:%d)", #call,               \
                                   cudaGetErrorString(e_), __FILE__, __LINE__);                \
    } while (0)

// Launch geometry: grid-stride kernels use a grid of `ctas_per_sm` CTAs
// on each SM.
// Workspaces size their per-CTA partial arrays for this many CTAs.
constexpr int kMaxGrid = 8 * 160;

inline int grid_for(const sscg_ctx* ctx, int64_t rows, int ctas_per_sm) {
    int64_t tiles = (rows + 255) / 256;
    int64_t g = (int64_t)ctx->sm_count * ctas_per_sm;
    if (tiles < g) g = tiles;
    if (g > kMaxGrid) g = kMaxGrid;
    return g < 1 ? 1 : (int)g;
}

// Persistent grid for a grid-stride kernel: as many CTAs as fit on the
// device at once (occupancy API), never more than there are row tiles.
template <class K>
inline int occupancy_grid(const sscg_ctx* ctx, K kernel, size_t smem, int64_t rows) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    return grid_for(ctx, rows, per_sm);
}

// Entries of a matrix row tile staged in shared memory: the largest tile's
// count plus 8 for the 16-byte widening of bulk copies, capped at 8192.
inline int stage_cap(const sscg_mat* m) {
    int cap = m->max_tile_nnz + 8;
    if (cap > 8192) cap = 8192;
    if (cap < 32) cap = 32;
    return (cap + 31) / 32 * 32;
}

// Kernel-family timing for SSCG_PROFILE: events on the context's stream
// around each launch, summed after the call for the steps actually taken.
enum { FAM_INIT = 0, FAM_MPK = 1, FAM_UPDATE = 2, FAM_DIR = 3, FAM_FINAL = 4, FAM_COUNT = 5 };

// Host side of a chunked launch loop.  After each chunk of launches the
// device word that says whether the solve has finished (a done flag, or a
// count of finished systems) is copied to a pinned slot behind an event; the
// host then waits on the event of the chunk kPollDepth - 1 chunks back, so up
// to kPollDepth chunks stay queued on the stream and a host-side stall shorter
// than kPollDepth - 1 chunks of device work leaves the GPU busy.  Chunks
// still queued when the device has finished return at their first
// instruction; that overshoot is as long as the protection (a depth of 3
// measured 4-5% slower on solves of a few milliseconds).  Uses pinned slots
// 0 .. kPollDepth - 1.
constexpr int kPollDepth = 2;

struct ChunkPoll {
    cudaEvent_t ev[kPollDepth];
    int made = 0;   // events created
    int chunk = 0;  // chunks recorded
    ChunkPoll() = default;
    ChunkPoll(const ChunkPoll&) = delete;
    ChunkPoll& operator=(const ChunkPoll&) = delete;
    ~ChunkPoll() {
        for (int i = 0; i < made; i++) cudaEventDestroy(ev[i]);
    }
    cudaError_t init() {
        for (; made < kPollDepth; made++) {
            const cudaError_t e = cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // Records the copy of *word after the chunk just launched.  Once a chunk
    // kPollDepth - 1 back exists, waits for it, sets *value to its word and
    // returns true; false otherwise.  *err: the error of the copy, record or wait.
    bool step(volatile int* pinned, const int* word, cudaStream_t st, int* value, cudaError_t* err) {
        const int slot = chunk % kPollDepth;
        cudaError_t e = cudaMemcpyAsync((void*)(pinned + slot), word, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[slot], st);
        *err = e;
        if (e != cudaSuccess) return false;
        const int old = chunk - (kPollDepth - 1);
        chunk++;
        if (old < 0) return false;
        e = cudaEventSynchronize(ev[old % kPollDepth]);
        *err = e;
        if (e != cudaSuccess) return false;
        *value = pinned[old % kPollDepth];
        return true;
    }
};

struct Prof {
    sscg_ctx* ctx;
    bool on;
    int used;
    int fam[65536];
    int step[65536];
    int64_t launches;
    explicit Prof(sscg_ctx* c, bool enable) : ctx(c), on(enable), used(0), launches(0) {}
    bool reserve(int pairs) {
        if (!on) return true;
        if (pairs > 65536) pairs = 65536;
        if (ctx->ev_cap >= 2 * pairs) return true;
        cudaEvent_t* nev = (cudaEvent_t*)realloc(ctx->ev, sizeof(cudaEvent_t) * 2 * pairs);
        if (!nev) return false;
        ctx->ev = nev;
        for (int i = ctx->ev_cap; i < 2 * pairs; i++)
            if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) return false;
        ctx->ev_cap = 2 * pairs;
        return true;
    }
    void begin() {
        if (on && 2 * used + 1 < ctx->ev_cap) cudaEventRecord(ctx->ev[2 * used], ctx->stream);
    }
    void end(int family, int k) {
        launches++;
        if (on && 2 * used + 1 < ctx->ev_cap) {
            cudaEventRecord(ctx->ev[2 * used + 1], ctx->stream);
            fam[used] = family;
            step[used] = k;
            used++;
        }
    }
    // Sum per family over launches whose step < steps_taken (init/final always).
    void collect(int steps_taken, double (&ms)[FAM_COUNT], int64_t (&cnt)[FAM_COUNT]) const {
        for (int f = 0; f < FAM_COUNT; f++) ms[f] = 0.0, cnt[f] = 0;
        if (!on) return;
        for (int i = 0; i < used; i++) {
            bool counted = fam[i] == FAM_INIT || fam[i] == FAM_FINAL || step[i] < steps_taken;
            if (!counted) continue;
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]) == cudaSuccess) {
                ms[fam[i]] += t;
                cnt[fam[i]]++;
            }
        }
    }
};

inline void fill_profile(sscg_info* info, const Prof& P, int steps_taken) {
    double ms[FAM_COUNT];
    int64_t cnt[FAM_COUNT];
    P.collect(steps_taken, ms, cnt);
    info->kernel_launches = P.launches;
    info->t_init_ms = ms[FAM_INIT];
    info->t_mpk_ms = ms[FAM_MPK];
    info->t_update_ms = ms[FAM_UPDATE];
    info->t_dir_ms = ms[FAM_DIR];
    info->t_final_ms = ms[FAM_FINAL];
    info->n_mpk = cnt[FAM_MPK];
    info->n_update = cnt[FAM_UPDATE];
    info->n_dir = cnt[FAM_DIR];
}

// Solvers (sstep.cu, pcg.cu)
int solve_sstep(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* opts,
                sscg_info* info, void* ws, size_t ws_bytes);
int sstep_workspace(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);
int solve_pcg(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* opts,
              sscg_info* info, void* ws, size_t ws_bytes);
int pcg_workspace(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);
int spmv_f64(sscg_ctx* ctx, const sscg_mat* mat, const double* x, double* y);
int gram_workspace(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);
int solve_gram(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* opts,
               sscg_info* info, void* ws, size_t ws_bytes, double blo, double bhi);
int bounds_workspace(const sscg_mat* mat, int steps, size_t* bytes);
int estimate_bounds(sscg_ctx* ctx, const sscg_mat* mat, int steps, const double* r0, void* ws, size_t ws_bytes,
                    double* lmin, double* lmax);
int splitmix_uniform(sscg_ctx* ctx, int64_t n, uint64_t seed, double* out);
int mixed_workspace(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);
int solve_mixed(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x, const sscg_opts* opts,
                sscg_info* info, void* ws, size_t ws_bytes, double blo, double bhi);

// Largest block size of a double-float solve in the monomial basis.  The
// monomial basis amplifies rounding with s (its Hankel moment matrix loses
// conditioning geometrically); with double-float's unit roundoff (2^-48,
// 32 times FP64's) the solution at s >= 7 drifts beyond 1e-7 of the FP64
// result on a 19^3 Poisson system (1.1e-7 at s = 8), so those solves take f64.
constexpr int kMaxSDf64Monomial = 6;

// Steps of the Lanczos estimate a Chebyshev-basis solve runs when the caller
// gives no basis interval, and the widening applied to its Ritz values.
constexpr int kAutoBoundSteps = 20;
constexpr double kAutoBoundLow = 0.95, kAutoBoundHigh = 1.05;

// The Lanczos estimate stops once ||r|| <= kLanczosTol ||r0||: the Krylov
// space is then invariant to working precision.  Past that point the
// double-float CG would square residuals below FP32's exponent range
// (rho underflows to 0) and put NaN coefficients into the tridiagonal.
constexpr double kLanczosTol = 1e-14;

// Spectral-bound network (mlp.cu): features pass plus inference.
size_t features_workspace();
int bounds_mlp(sscg_ctx* ctx, const sscg_mat* m, int h, const double* model, void* ws, size_t ws_bytes, double* lmin,
               double* lmax);

}  // namespace sscg
