// C-ABI entry points of libsscg: context, matrix, preconditioner, solves.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "spmv.cuh"

using namespace sscg;

namespace {

// Flags gathered by the analysis kernel.
struct Analysis {
    unsigned long long bad_col;
    unsigned long long nonfinite;
    unsigned long long not_exact;
    unsigned long long nonpos_diag;
    unsigned long long bandwidth;
    unsigned long long dmin_bits;  // positive doubles order like their bit patterns
    unsigned long long dmax_bits;
    unsigned dia_bad;  // entries violating the constant-coefficient diagonal form
    unsigned pad;
    unsigned long long out_of_f32;  // nonzero values outside FP32's normal range (|v| > FLT_MAX or < FLT_MIN)
};

// Per row: check column range and finiteness, split values into FP32
// hi + lo, sum the diagonal, record bandwidth, build 1/diag in FP64 and DF64.
__global__ void __launch_bounds__(kThreads) k_analyze(int n, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val, float* __restrict__ vhi,
                                                      float* __restrict__ vlo, double* __restrict__ diag,
                                                      double* __restrict__ dinv, float2* __restrict__ dinv_df,
                                                      float2* __restrict__ diag_df, float* __restrict__ dinv_f,
                                                      Analysis* out) {
    __shared__ unsigned long long s_bad, s_nf, s_ne, s_np, s_bw, s_mn, s_mx, s_or;
    if (threadIdx.x == 0) {
        s_bad = s_nf = s_ne = s_np = s_bw = s_or = 0ull;
        s_mn = ~0ull;
        s_mx = 0ull;
    }
    __syncthreads();
    unsigned long long bad = 0, nf = 0, ne = 0, np = 0, bw = 0, mn = ~0ull, mx = 0ull, orr = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int c = col[k];
            double v = val[k];
            if (c < 0 || c >= n) bad++;
            if (!isfinite(v)) nf++;
            const double av = fabs(v);
            if (av != 0.0 && (av > 3.4028234663852886e38 || av < 1.1754943508222875e-38)) orr++;
            float hi = __double2float_rn(v);
            float lo = __double2float_rn(v - (double)hi);
            vhi[k] = hi;
            vlo[k] = lo;
            if ((double)hi != v) ne++;
            unsigned long long dist = (unsigned long long)(c > i ? c - i : i - c);
            bw = dist > bw ? dist : bw;
            if (c == i) d += v;
        }
        diag[i] = d;
        {
            float dh = __double2float_rn(d);
            diag_df[i] = make_float2(dh, __double2float_rn(d - (double)dh));
        }
        if (!(d > 0.0) || !isfinite(d)) {
            np++;
            dinv[i] = 0.0;
            dinv_df[i] = make_float2(0.f, 0.f);
            dinv_f[i] = 0.f;
        } else {
            double inv = 1.0 / d;
            dinv[i] = inv;
            float hi = __double2float_rn(inv);
            dinv_df[i] = make_float2(hi, __double2float_rn(inv - (double)hi));
            dinv_f[i] = hi;
            unsigned long long bits = (unsigned long long)__double_as_longlong(d);
            mn = bits < mn ? bits : mn;
            mx = bits > mx ? bits : mx;
        }
    }
    if (bad) atomicAdd(&s_bad, bad);
    if (nf) atomicAdd(&s_nf, nf);
    if (ne) atomicAdd(&s_ne, ne);
    if (orr) atomicAdd(&s_or, orr);
    if (np) atomicAdd(&s_np, np);
    atomicMax(&s_bw, bw);
    atomicMin(&s_mn, mn);
    atomicMax(&s_mx, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_bad) atomicAdd(&out->bad_col, s_bad);
        if (s_nf) atomicAdd(&out->nonfinite, s_nf);
        if (s_ne) atomicAdd(&out->not_exact, s_ne);
        if (s_or) atomicAdd(&out->out_of_f32, s_or);
        if (s_np) atomicAdd(&out->nonpos_diag, s_np);
        atomicMax(&out->bandwidth, s_bw);
        atomicMin(&out->dmin_bits, s_mn);
        atomicMax(&out->dmax_bits, s_mx);
    }
}

struct DiaDesc {
    int k;
    int off[kDiaMax];  // ascending
    double c[kDiaMax];
};

// Check the constant-coefficient diagonal form: every entry (i, j) has
// j - i equal to one of the offsets and the value of that offset; no offset
// twice in a row.  Writes the presence mask of every row; any violation sets
// *bad.
__global__ void __launch_bounds__(kThreads) k_dia_check(int n, const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ val, DiaDesc d,
                                                        uint32_t* __restrict__ mask, unsigned* bad) {
    __shared__ long long s_off[kDiaMax];
    __shared__ double s_c[kDiaMax];
    for (int t = threadIdx.x; t < d.k; t += blockDim.x) {
        s_off[t] = d.off[t];
        s_c[t] = d.c[t];
    }
    __syncthreads();
    unsigned nbad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t m = 0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            const long long o = (long long)col[k] - i;
            int lo = 0, hi = d.k - 1, t = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] == o) {
                    t = mid;
                    break;
                }
                if (s_off[mid] < o) lo = mid + 1;
                else hi = mid - 1;
            }
            if (t < 0 || ((m >> t) & 1u) || val[k] != s_c[t]) {
                nbad++;
                continue;
            }
            m |= 1u << t;
        }
        mask[i] = m;
    }
    if (nbad) atomicAdd(bad, nbad);
}

struct MatLayout {
    int32_t* rowptr;
    int32_t* col;
    double* val;
    float* vhi;
    float* vlo;
    double* diag;
    double* dinv;
    float2* dinv_df;
    float2* diag_df;
    float* dinv_f;
    uint32_t* mask;
    Analysis* an;
    size_t bytes;
};

MatLayout mat_layout(int64_t n, int64_t nnz, void* base) {
    MatLayout L;
    Carve c(base, base ? ~(size_t)0 : 0);
    // +16 entries of slack after every entry array so vector loads of a
    // tile's range never leave the allocation.
    L.rowptr = c.take<int32_t>((size_t)n + 1 + 16);
    L.col = c.take<int32_t>((size_t)nnz + 16);
    L.val = c.take<double>((size_t)nnz + 16);
    L.vhi = c.take<float>((size_t)nnz + 16);
    L.vlo = c.take<float>((size_t)nnz + 16);
    L.diag = c.take<double>((size_t)n + 16);
    L.dinv = c.take<double>((size_t)n + 16);
    L.dinv_df = c.take<float2>((size_t)n + 16);
    L.diag_df = c.take<float2>((size_t)n + 16);
    L.dinv_f = c.take<float>((size_t)n + 16);
    L.mask = c.take<uint32_t>((size_t)n + 16);
    L.an = c.take<Analysis>(1);
    L.bytes = c.used;
    return L;
}

// Try the constant-coefficient diagonal form: take the offsets and values
// of the densest row (row i0, its entries from position k0), require them
// FP32-exact with a positive diagonal, and check every row on the device.
int detect_dia(sscg_ctx* ctx, sscg_mat* m, uint32_t* mask, Analysis* an, int32_t k0, int64_t i0, int len) {
    cudaStream_t st = ctx->stream;
    std::vector<int32_t> c((size_t)len);
    std::vector<double> v((size_t)len);
    SSCG_CUDA(ctx, cudaMemcpyAsync(c.data(), m->col + k0, len * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaMemcpyAsync(v.data(), m->val + k0, len * sizeof(double), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<std::pair<long long, double>> e;
    for (int t = 0; t < len; t++) e.push_back({(long long)c[t] - i0, v[t]});
    std::sort(e.begin(), e.end());
    DiaDesc d;
    memset(&d, 0, sizeof(d));
    d.k = len;
    int diag_t = -1;
    for (int t = 0; t < len; t++) {
        if (t > 0 && e[t].first == e[t - 1].first) return SSCG_OK;       // duplicate entry: keep CSR
        if ((double)(float)e[t].second != e[t].second) return SSCG_OK;  // not FP32-exact
        if (e[t].first < INT32_MIN || e[t].first > INT32_MAX) return SSCG_OK;
        d.off[t] = (int)e[t].first;
        d.c[t] = e[t].second;
        if (e[t].first == 0) diag_t = t;
    }
    if (diag_t < 0 || !(d.c[diag_t] > 0.0)) return SSCG_OK;
    SSCG_CUDA(ctx, cudaMemsetAsync(&an->dia_bad, 0, sizeof(unsigned), st));
    k_dia_check<<<grid_for(ctx, m->n, 4), kThreads, 0, st>>>((int)m->n, m->rowptr, m->col, m->val, d, mask,
                                                             &an->dia_bad);
    SSCG_CUDA(ctx, cudaGetLastError());
    unsigned bad = 1;
    SSCG_CUDA(ctx, cudaMemcpyAsync(&bad, &an->dia_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    if (bad != 0) return SSCG_OK;
    m->dia = 1;
    m->dia_k = d.k;
    for (int t = 0; t < d.k; t++) {
        m->dia_off[t] = d.off[t];
        m->dia_c[t] = d.c[t];
    }
    m->dia_mask = mask;
    m->dia_d = d.c[diag_t];
    m->dia_dinv = 1.0 / d.c[diag_t];
    m->dia_cen = diag_t;
    m->dia_lap = 1;
    m->dia_co = 0.0;
    m->dia_reach = 0;
    for (int t = 0; t < d.k; t++) {
        m->dia_reach = std::max<int64_t>(m->dia_reach, std::abs((int64_t)d.off[t]));
        if (t == diag_t) continue;
        if (m->dia_co == 0.0) m->dia_co = d.c[t];
        else if (d.c[t] != m->dia_co) m->dia_lap = 0;
    }
    if (m->dia_co == 0.0) m->dia_lap = 0;
    return SSCG_OK;
}

}  // namespace

extern "C" {

int sscg_version(void) { return 100; }

const char* sscg_status_str(int s) {
    switch (s) {
        case SSCG_OK: return "converged";
        case SSCG_NOT_CONVERGED: return "not converged within maxit";
        case SSCG_BREAKDOWN: return "breakdown (singular or indefinite s x s system, or non-finite value)";
        case SSCG_TIMEOUT: return "bounded device wait timed out";
        case SSCG_ERR_INVALID: return "invalid argument";
        case SSCG_ERR_NOT_SPD: return "matrix has a non-positive or missing diagonal entry";
        case SSCG_ERR_CUDA: return "CUDA error";
        case SSCG_ERR_SPACE: return "storage or workspace too small or misaligned";
        case SSCG_ERR_NONFINITE: return "non-finite input";
        default: return "unknown status";
    }
}

int sscg_create(sscg_ctx** out, void* stream) {
    if (!out) return SSCG_ERR_INVALID;
    *out = nullptr;
    sscg_ctx* c = (sscg_ctx*)calloc(1, sizeof(sscg_ctx));
    if (!c) return SSCG_ERR_INVALID;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    int major = 0, minor = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
    if (e == cudaSuccess && !(major == 10 && minor == 3)) {
        free(c);
        return SSCG_ERR_CUDA;  // the library holds sm_103a code only
    }
    void* pinned = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc(&pinned, 64, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        free(c);
        return SSCG_ERR_CUDA;
    }
    memset(pinned, 0, 64);
    c->pinned = (volatile int*)pinned;
    *out = c;
    return SSCG_OK;
}

int sscg_destroy(sscg_ctx* c) {
    if (!c) return SSCG_ERR_INVALID;
    if (c->pinned) cudaFreeHost((void*)c->pinned);
    for (int i = 0; i < c->ev_cap; i++) cudaEventDestroy(c->ev[i]);
    free(c->ev);
    free(c);
    return SSCG_OK;
}

const char* sscg_last_error(const sscg_ctx* c) { return c ? c->err : "null context"; }

int sscg_mat_storage_bytes(int64_t n, int64_t nnz, size_t* bytes) {
    if (!bytes || n <= 0 || n >= INT32_MAX || nnz < 0 || nnz >= INT32_MAX - 64) return SSCG_ERR_INVALID;
    *bytes = mat_layout(n, nnz, nullptr).bytes;
    return SSCG_OK;
}

int sscg_mat_create_csr(sscg_ctx* ctx, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                        const double* val, unsigned flags, void* storage, size_t storage_bytes, sscg_mat** out) {
    if (!ctx || !out) return SSCG_ERR_INVALID;
    *out = nullptr;
    size_t need = 0;
    if (sscg_mat_storage_bytes(n, nnz, &need) != SSCG_OK)
        return set_err(ctx, SSCG_ERR_INVALID, "n = %lld, nnz = %lld out of range", (long long)n, (long long)nnz);
    if (!rowptr || (nnz > 0 && (!colind || !val))) return set_err(ctx, SSCG_ERR_INVALID, "null CSR array");
    if (!storage || storage_bytes < need || ((uintptr_t)storage & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "matrix storage needs %zu bytes, 256-byte aligned", need);
    cudaStream_t st = ctx->stream;
    MatLayout L = mat_layout(n, nnz, storage);
    const cudaMemcpyKind kind = (flags & SSCG_HOST_ARRAYS) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    SSCG_CUDA(ctx, cudaMemcpyAsync(L.rowptr, rowptr, (n + 1) * sizeof(int32_t), kind, st));
    SSCG_CUDA(ctx, cudaMemsetAsync(L.rowptr + n + 1, 0, 16 * sizeof(int32_t), st));
    if (nnz > 0) {
        SSCG_CUDA(ctx, cudaMemcpyAsync(L.col, colind, nnz * sizeof(int32_t), kind, st));
        SSCG_CUDA(ctx, cudaMemcpyAsync(L.val, val, nnz * sizeof(double), kind, st));
    }
    SSCG_CUDA(ctx, cudaMemsetAsync(L.col + nnz, 0, 16 * sizeof(int32_t), st));
    SSCG_CUDA(ctx, cudaMemsetAsync(L.val + nnz, 0, 16 * sizeof(double), st));
    SSCG_CUDA(ctx, cudaMemsetAsync(L.vhi + nnz, 0, 16 * sizeof(float), st));
    SSCG_CUDA(ctx, cudaMemsetAsync(L.vlo + nnz, 0, 16 * sizeof(float), st));
    // Row pointers are checked on the host: monotone, 0 .. nnz.
    std::vector<int32_t> hr((size_t)n + 1);
    SSCG_CUDA(ctx, cudaMemcpyAsync(hr.data(), L.rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    if (hr[0] != 0 || hr[(size_t)n] != nnz)
        return set_err(ctx, SSCG_ERR_INVALID, "rowptr[0] must be 0 and rowptr[n] must be nnz");
    int max_row = 0, max_tile = 0;
    int64_t max_row_at = 0;
    for (int64_t i = 0; i < n; i++) {
        int len = hr[i + 1] - hr[i];
        if (len < 0) return set_err(ctx, SSCG_ERR_INVALID, "rowptr decreases at row %lld", (long long)i);
        if (len > max_row) {
            max_row = len;
            max_row_at = i;
        }
    }
    for (int64_t t = 0; t < n; t += kTileRows) {
        int64_t e = std::min<int64_t>(n, t + kTileRows);
        max_tile = std::max(max_tile, hr[e] - hr[t]);
    }
    Analysis a0;
    memset(&a0, 0, sizeof(a0));
    a0.dmin_bits = ~0ull;
    SSCG_CUDA(ctx, cudaMemcpyAsync(L.an, &a0, sizeof(a0), cudaMemcpyHostToDevice, st));
    int G = grid_for(ctx, n, 4);
    k_analyze<<<G, kThreads, 0, st>>>((int)n, L.rowptr, L.col, L.val, L.vhi, L.vlo, L.diag, L.dinv, L.dinv_df,
                                      L.diag_df, L.dinv_f, L.an);
    SSCG_CUDA(ctx, cudaGetLastError());
    Analysis a;
    SSCG_CUDA(ctx, cudaMemcpyAsync(&a, L.an, sizeof(a), cudaMemcpyDeviceToHost, st));
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    if (a.bad_col) return set_err(ctx, SSCG_ERR_INVALID, "%llu column indices outside [0, n)", a.bad_col);
    if (a.nonfinite) return set_err(ctx, SSCG_ERR_NONFINITE, "%llu non-finite matrix values", a.nonfinite);
    if (a.nonpos_diag)
        return set_err(ctx, SSCG_ERR_NOT_SPD, "%llu rows with a non-positive or missing diagonal", a.nonpos_diag);
    sscg_mat* m = (sscg_mat*)calloc(1, sizeof(sscg_mat));
    if (!m) return set_err(ctx, SSCG_ERR_INVALID, "out of host memory");
    m->n = n;
    m->nnz = nnz;
    m->rowptr = L.rowptr;
    m->col = L.col;
    m->val = L.val;
    m->vhi = L.vhi;
    m->vlo = L.vlo;
    m->diag = L.diag;
    m->dinv = L.dinv;
    m->dinv_df = L.dinv_df;
    m->dinv_f = L.dinv_f;
    m->diag_df = L.diag_df;
    m->bandwidth = (int64_t)a.bandwidth;
    m->exact_fp32 = a.not_exact == 0;
    m->out_of_f32 = a.out_of_f32 != 0;
    m->max_row_nnz = max_row;
    m->max_tile_nnz = max_tile;
    double dmn, dmx;
    memcpy(&dmn, &a.dmin_bits, 8);
    memcpy(&dmx, &a.dmax_bits, 8);
    m->dmin = dmn;
    m->dmax = dmx;
    m->prec = SSCG_PREC_JACOBI;
    if (!(flags & SSCG_MAT_CSR_ONLY) && max_row > 0 && max_row <= kDiaMax) {
        if (int e = detect_dia(ctx, m, L.mask, L.an, hr[(size_t)max_row_at], max_row_at, max_row)) {
            free(m);
            return e;
        }
    }
    *out = m;
    return SSCG_OK;
}

int sscg_mat_destroy(sscg_mat* m) {
    if (!m) return SSCG_ERR_INVALID;
    free(m);
    return SSCG_OK;
}

int sscg_mat_props_get(const sscg_mat* m, sscg_mat_props* p) {
    if (!m || !p) return SSCG_ERR_INVALID;
    p->n = m->n;
    p->nnz = m->nnz;
    p->bandwidth = m->bandwidth;
    p->values_exact_fp32 = m->exact_fp32;
    p->max_row_nnz = m->max_row_nnz;
    p->diag_min = m->dmin;
    p->diag_max = m->dmax;
    p->prec = m->prec;
    p->prec_degree = m->degree;
    p->prec_lmin = m->plmin;
    p->prec_lmax = m->plmax;
    p->format = m->dia ? SSCG_FORMAT_DIA_CONST : SSCG_FORMAT_CSR;
    p->dia_offsets = m->dia ? m->dia_k : 0;
    return SSCG_OK;
}

int sscg_set_preconditioner(sscg_mat* m, int prec, int degree, double lmin, double lmax) {
    if (!m) return SSCG_ERR_INVALID;
    if (prec == SSCG_PREC_NONE || prec == SSCG_PREC_JACOBI) {
        m->prec = prec;
        m->degree = 0;
        m->plmin = m->plmax = 0.0;
        return SSCG_OK;
    }
    if (prec == SSCG_PREC_CHEB) {
        if (degree < 1 || degree > 64 || !(lmin > 0.0) || !(lmax > lmin) || !std::isfinite(lmax))
            return SSCG_ERR_INVALID;
        m->prec = prec;
        m->degree = degree;
        m->plmin = lmin;
        m->plmax = lmax;
        return SSCG_OK;
    }
    return SSCG_ERR_INVALID;
}

// The moment recurrence of Algorithm 6 serves the monomial basis with a
// diagonal preconditioner; every other combination forms the Gram blocks.
static bool use_gram(const sscg_mat* m, const sscg_opts* o) {
    return o->basis != SSCG_BASIS_MONOMIAL || m->prec == SSCG_PREC_CHEB || (o->flags & SSCG_DIRECT_GRAM);
}

static bool auto_bounds(const sscg_opts* o) {
    return o->basis != SSCG_BASIS_MONOMIAL && o->basis_lmin == 0.0 && o->basis_lmax == 0.0;
}

// The network predicts the interval of D^-1 A, which is the operator of the
// basis only under the Jacobi preconditioner.
static bool model_bounds(const sscg_mat* m) { return m->bounds_model && m->prec == SSCG_PREC_JACOBI; }

int sscg_solve_workspace_bytes(const sscg_mat* m, const sscg_opts* o, size_t* bytes) {
    if (!m || !o || !bytes || o->s < 1 || o->s > kMaxS || o->maxit < 0) return SSCG_ERR_INVALID;
    if (o->arith != SSCG_ARITH_MIXED && !use_gram(m, o)) return sstep_workspace(m, o, bytes);
    if (o->arith == SSCG_ARITH_MIXED) mixed_workspace(m, o, bytes);
    else gram_workspace(m, o, bytes);
    if (auto_bounds(o)) {
        size_t bb = 0;
        if (model_bounds(m)) bb = features_workspace();
        else bounds_workspace(m, kAutoBoundSteps, &bb);
        *bytes = std::max(*bytes, bb);
    }
    return SSCG_OK;
}

static int solve_once(sscg_ctx* ctx, const sscg_mat* m, const double* b, double* x, const sscg_opts* o,
                      sscg_info* info, void* ws, size_t ws_bytes) {
    if (!m || !o || !b || !x) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    if (o->s < 1 || o->s > kMaxS) return set_err(ctx, SSCG_ERR_INVALID, "s = %d outside 1..%d", o->s, kMaxS);
    if (o->maxit < 0 || !(o->tol >= 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad maxit or tol");
    if (o->basis != SSCG_BASIS_MONOMIAL && o->basis != SSCG_BASIS_CHEBYSHEV && o->basis != SSCG_BASIS_NEWTON)
        return set_err(ctx, SSCG_ERR_INVALID, "unknown basis %d", o->basis);
    if (o->arith != SSCG_ARITH_F64 && o->arith != SSCG_ARITH_DF64 && o->arith != SSCG_ARITH_MIXED)
        return set_err(ctx, SSCG_ERR_INVALID, "arith %d not supported", o->arith);
    if (o->arith == SSCG_ARITH_MIXED && m->prec == SSCG_PREC_CHEB)
        return set_err(ctx, SSCG_ERR_INVALID, "the mixed-precision mode takes a diagonal preconditioner");
    if (o->arith != SSCG_ARITH_F64 && m->out_of_f32)
        return set_err(ctx, SSCG_ERR_INVALID, "matrix values lie outside FP32's normal range, which double-float "
                                              "and mixed arithmetic carry; use f64");
    if (o->arith == SSCG_ARITH_DF64 && o->basis == SSCG_BASIS_MONOMIAL && o->s > kMaxSDf64Monomial)
        return set_err(ctx, SSCG_ERR_INVALID, "double-float arithmetic takes the monomial basis up to s = %d; use f64",
                       kMaxSDf64Monomial);
    if (o->arith != SSCG_ARITH_MIXED && !use_gram(m, o)) return solve_sstep(ctx, m, b, x, o, info, ws, ws_bytes);
    double lo = o->basis_lmin, hi = o->basis_lmax;
    if (auto_bounds(o)) {
        size_t need = 0;
        sscg_solve_workspace_bytes(m, o, &need);
        if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
            return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned", need);
        int rc = model_bounds(m) ? bounds_mlp(ctx, m, m->bounds_h, m->bounds_model, ws, ws_bytes, &lo, &hi)
                                 : estimate_bounds(ctx, m, kAutoBoundSteps, nullptr, ws, ws_bytes, &lo, &hi);
        if (rc != SSCG_OK) return rc;
        lo *= kAutoBoundLow;
        hi *= kAutoBoundHigh;
    }
    if (o->basis != SSCG_BASIS_MONOMIAL && !(hi > lo && lo >= 0.0))
        return set_err(ctx, SSCG_ERR_INVALID, "Chebyshev and Newton bases need 0 <= basis_lmin < basis_lmax");
    if (o->arith == SSCG_ARITH_MIXED) return solve_mixed(ctx, m, b, x, o, info, ws, ws_bytes, lo, hi);
    return solve_gram(ctx, m, b, x, o, info, ws, ws_bytes, lo, hi);
}

// Adaptive block size (Section IV lists adaptive s among the remedies for
// the s-step basis's loss of independence): a solve that breaks down leaves
// x at its last good iterate; it is restarted from there with s halved, on
// the CG steps left of the budget maxit * s, until it converges, stops for
// another reason, or breaks down at s = 1.  The history concatenates the
// segments (each restart's first entry, its true initial residual, replaces
// the previous segment's last one).
int sscg_solve(sscg_ctx* ctx, const sscg_mat* m, const double* b, double* x, const sscg_opts* o, sscg_info* info,
               void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (!o || !(o->flags & SSCG_ADAPTIVE_S)) {
        const int rc = solve_once(ctx, m, b, x, o, info, ws, ws_bytes);
        if (info && rc >= 0) info->s_final = o->s;
        return rc;
    }
    sscg_opts cur = *o;
    cur.flags &= ~SSCG_ADAPTIVE_S;
    int64_t budget = (int64_t)o->maxit * o->s;  // CG steps
    sscg_info tot;
    memset(&tot, 0, sizeof(tot));
    int used = 0;  // history entries written
    for (;;) {
        cur.maxit = (int)std::min<int64_t>(INT32_MAX, (budget + cur.s - 1) / cur.s);
        sscg_info seg;
        memset(&seg, 0, sizeof(seg));
        if (info && info->hist && info->hist_cap > 0) {
            const int at = used > 0 ? used - 1 : 0;
            seg.hist = info->hist + at;
            seg.hist_cap = info->hist_cap - at;
        }
        const int rc = solve_once(ctx, m, b, x, &cur, &seg, ws, ws_bytes);
        if (rc < 0) return rc;
        tot.outer_iters += seg.outer_iters;
        tot.equiv_iters += seg.equiv_iters;
        tot.kernel_launches += seg.kernel_launches;
        tot.t_init_ms += seg.t_init_ms, tot.t_mpk_ms += seg.t_mpk_ms, tot.t_update_ms += seg.t_update_ms;
        tot.t_dir_ms += seg.t_dir_ms, tot.t_final_ms += seg.t_final_ms;
        tot.n_mpk += seg.n_mpk, tot.n_update += seg.n_update, tot.n_dir += seg.n_dir;
        if (seg.hist) used = (int)(seg.hist - info->hist) + seg.hist_len;
        budget -= seg.equiv_iters;
        if (rc != SSCG_BREAKDOWN || cur.s == 1 || budget <= 0) {
            if (info) {
                double* h = info->hist;
                const int cap = info->hist_cap;
                *info = tot;
                info->hist = h;
                info->hist_cap = cap;
                info->hist_len = h ? used : 0;
                info->status = rc;
                info->rel_res_recursive = seg.rel_res_recursive;
                info->rel_res_true = seg.rel_res_true;
                info->s_final = cur.s;
            }
            return rc;
        }
        cur.s = std::max(1, cur.s / 2);
    }
}

int sscg_bounds_workspace_bytes(const sscg_mat* m, int steps, size_t* bytes) {
    if (!m || !bytes || steps < 1 || steps > 100000) return SSCG_ERR_INVALID;
    return bounds_workspace(m, steps, bytes);
}

int sscg_estimate_bounds(sscg_ctx* ctx, const sscg_mat* m, int steps, const double* r0, void* ws, size_t ws_bytes,
                         double* lmin, double* lmax) {
    if (!ctx) return SSCG_ERR_INVALID;
    return estimate_bounds(ctx, m, steps, r0, ws, ws_bytes, lmin, lmax);
}

int sscg_uniform(sscg_ctx* ctx, int64_t n, uint64_t seed, double* out) {
    if (!ctx) return SSCG_ERR_INVALID;
    return splitmix_uniform(ctx, n, seed, out);
}

int sscg_pcg_workspace_bytes(const sscg_mat* m, const sscg_opts* o, size_t* bytes) {
    if (!m || !o || !bytes || o->maxit < 0) return SSCG_ERR_INVALID;
    return pcg_workspace(m, o, bytes);
}

int sscg_pcg_solve(sscg_ctx* ctx, const sscg_mat* m, const double* b, double* x, const sscg_opts* o, sscg_info* info,
                   void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (m && o && o->arith != SSCG_ARITH_F64 && m->out_of_f32)
        return set_err(ctx, SSCG_ERR_INVALID, "matrix values lie outside FP32's normal range, which double-float "
                                              "arithmetic carries; use f64");
    return solve_pcg(ctx, m, b, x, o, info, ws, ws_bytes);
}

int sscg_spmv(sscg_ctx* ctx, const sscg_mat* m, const double* x, double* y) {
    if (!ctx || !m || !x || !y) return SSCG_ERR_INVALID;
    return spmv_f64(ctx, m, x, y);
}

}  // extern "C"

namespace sscg {

__global__ void __launch_bounds__(kThreads) k_spmv_f64(MatView M, const double* __restrict__ x, double* __restrict__ y) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_rp[kTileRows + 1];
    const int ntiles = (M.n + kTileRows - 1) / kTileRows;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        double v;
        int row;
        if (tile_spmv<ArithF64, VAL_F64>(M, tile, [&](int c) { return __ldg(x + c); }, v, row, smem, s_rp)) y[row] = v;
    }
}

int spmv_f64(sscg_ctx* ctx, const sscg_mat* m, const double* x, double* y) {
    const int cap = stage_cap(m);
    MatView M{};
    M.n = (int)m->n;
    M.cap = cap;
    M.rowptr = m->rowptr;
    M.col = m->col;
    M.val = m->val;
    M.vhi = m->vhi;
    M.vlo = m->vlo;
    size_t smem = stage_bytes<ArithF64, VAL_F64>(cap);
    SSCG_CUDA(ctx, cudaFuncSetAttribute(k_spmv_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_spmv_f64<<<grid_for(ctx, m->n, 8), kThreads, smem, ctx->stream>>>(M, x, y);
    SSCG_CUDA(ctx, cudaGetLastError());
    return SSCG_OK;
}

}  // namespace sscg
