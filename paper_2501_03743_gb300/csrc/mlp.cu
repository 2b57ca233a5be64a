// Spectral-bound network: a small multilayer perceptron that maps features
// of a matrix to (ln lambda_min, ln lambda_max) of D^-1 A, the interval the
// Chebyshev basis of Section IV needs (the paper does not say where the
// bounds come from).  Training and inference run on the device in FP64:
// with about 5,000 parameters the network is far too small for the tensor
// cores to matter, and FP64 keeps the gradients comparable with an FP64
// reference to rounding.
//
//   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3
//   parameters packed as [W1 (h x d, row-major), b1, W2 (h x h), b2, W3 (o x h), b3]
//   loss = mean over batch and outputs of (y - t)^2
//
// Every reduction over the batch runs in a fixed order, so training is
// deterministic.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace sscg {

namespace {

struct MlpDims {
    int d, h, o;
    int64_t np() const { return (int64_t)h * d + h + (int64_t)h * h + h + (int64_t)o * h + o; }
};

// out[b][u] = act(bias[u] + sum_k W[u][k] in[b][k]); act = tanh or identity.
__global__ void __launch_bounds__(kThreads) k_dense_fwd(int B, int nin, int nout, const double* __restrict__ W,
                                                        const double* __restrict__ bias, const double* __restrict__ in,
                                                        double* __restrict__ out, int act_tanh) {
    const int64_t total = (int64_t)B * nout;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / nout), u = (int)(e % nout);
        const double* w = W + (size_t)u * nin;
        const double* x = in + (size_t)b * nin;
        double t = bias[u];
        for (int k = 0; k < nin; k++) t = fma(w[k], x[k], t);
        out[e] = act_tanh ? tanh(t) : t;
    }
}

// dY = 2 (Y - T) / (B o): the gradient of the mean squared error.
__global__ void __launch_bounds__(kThreads) k_out_grad(int64_t total, double scale, const double* __restrict__ Y,
                                                       const double* __restrict__ T, double* __restrict__ dY) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        dY[e] = 2.0 * (Y[e] - T[e]) * scale;
}

// Back through a dense layer into the tanh layer below it:
// dZprev[b][k] = (sum_u W[u][k] dZ[b][u]) (1 - Aprev[b][k]^2).
__global__ void __launch_bounds__(kThreads) k_dense_bwd_data(int B, int nin, int nout, const double* __restrict__ W,
                                                             const double* __restrict__ dZ,
                                                             const double* __restrict__ Aprev,
                                                             double* __restrict__ dZprev) {
    const int64_t total = (int64_t)B * nin;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / nin), k = (int)(e % nin);
        const double* dz = dZ + (size_t)b * nout;
        double t = 0.0;
        for (int u = 0; u < nout; u++) t = fma(W[(size_t)u * nin + k], dz[u], t);
        const double a = Aprev[e];
        dZprev[e] = t * (1.0 - a * a);
    }
}

// Weight and bias gradients of a dense layer: gW[u][k] = sum_b dZ[b][u]
// Aprev[b][k], gbias[u] = sum_b dZ[b][u].  One warp per parameter, lanes
// striding the batch, then a fixed shuffle tree (deterministic).
__global__ void __launch_bounds__(kThreads) k_dense_bwd_w(int B, int nin, int nout, const double* __restrict__ dZ,
                                                          const double* __restrict__ Aprev, double* __restrict__ gW,
                                                          double* __restrict__ gbias) {
    const int lane = threadIdx.x & 31;
    const int total = nout * nin + nout;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < total; e += nwarps) {
        double t = 0.0;
        if (e < nout * nin) {
            const int u = e / nin, k = e % nin;
            for (int b = lane; b < B; b += 32) t = fma(dZ[(size_t)b * nout + u], Aprev[(size_t)b * nin + k], t);
        } else {
            const int u = e - nout * nin;
            for (int b = lane; b < B; b += 32) t += dZ[(size_t)b * nout + u];
        }
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
        if (lane == 0) {
            if (e < nout * nin) gW[e] = t;
            else gbias[e - nout * nin] = t;
        }
    }
}

// Mean squared error by one CTA in a fixed order.
__global__ void __launch_bounds__(kThreads) k_mse(int64_t total, const double* __restrict__ Y,
                                                  const double* __restrict__ T, double* __restrict__ out) {
    __shared__ double sh[kThreads / 32];
    double t = 0.0;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const double d = Y[e] - T[e];
        t = fma(d, d, t);
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
        *out = s / (double)total;
    }
}

// Adam (Kingma and Ba, 2015) with the bias corrections c1 = 1 - b1^t and
// c2 = 1 - b2^t of step t.
__global__ void __launch_bounds__(kThreads) k_adam(int64_t np, double* __restrict__ theta,
                                                   const double* __restrict__ g, double* __restrict__ m,
                                                   double* __restrict__ v, double lr, double b1, double b2, double eps,
                                                   double c1, double c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const double gi = g[i];
        const double mi = b1 * m[i] + (1.0 - b1) * gi;
        const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
    }
}

struct MlpWork {
    double *H1, *H2, *Y, *dY, *dZ2, *dZ1, *grad, *m, *v, *loss;
    size_t bytes;
};

MlpWork mlp_plan(const MlpDims& D, int B, void* base) {
    MlpWork w{};
    Carve c(base, 0);
    w.H1 = c.take<double>((size_t)B * D.h);
    w.H2 = c.take<double>((size_t)B * D.h);
    w.Y = c.take<double>((size_t)B * D.o);
    w.dY = c.take<double>((size_t)B * D.o);
    w.dZ2 = c.take<double>((size_t)B * D.h);
    w.dZ1 = c.take<double>((size_t)B * D.h);
    w.grad = c.take<double>((size_t)D.np());
    w.m = c.take<double>((size_t)D.np());
    w.v = c.take<double>((size_t)D.np());
    w.loss = c.take<double>(1);
    w.bytes = c.used;
    return w;
}

int grid_n(const sscg_ctx* ctx, int64_t threads) {
    const int64_t g = (threads + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)ctx->sm_count * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

void launch_forward(const sscg_ctx* ctx, const MlpDims& D, const double* th, int B, const double* X,
                    const MlpWork& w) {
    cudaStream_t st = ctx->stream;
    const double* W1 = th;
    const double* b1 = W1 + (size_t)D.h * D.d;
    const double* W2 = b1 + D.h;
    const double* b2 = W2 + (size_t)D.h * D.h;
    const double* W3 = b2 + D.h;
    const double* b3 = W3 + (size_t)D.o * D.h;
    k_dense_fwd<<<grid_n(ctx, (int64_t)B * D.h), kThreads, 0, st>>>(B, D.d, D.h, W1, b1, X, w.H1, 1);
    k_dense_fwd<<<grid_n(ctx, (int64_t)B * D.h), kThreads, 0, st>>>(B, D.h, D.h, W2, b2, w.H1, w.H2, 1);
    k_dense_fwd<<<grid_n(ctx, (int64_t)B * D.o), kThreads, 0, st>>>(B, D.h, D.o, W3, b3, w.H2, w.Y, 0);
}

void launch_backward(const sscg_ctx* ctx, const MlpDims& D, const double* th, int B, const double* X,
                     const double* T, const MlpWork& w, double* grad) {
    cudaStream_t st = ctx->stream;
    const double* W2 = th + (size_t)D.h * D.d + D.h;
    const double* W3 = W2 + (size_t)D.h * D.h + D.h;
    double* gW1 = grad;
    double* gb1 = gW1 + (size_t)D.h * D.d;
    double* gW2 = gb1 + D.h;
    double* gb2 = gW2 + (size_t)D.h * D.h;
    double* gW3 = gb2 + D.h;
    double* gb3 = gW3 + (size_t)D.o * D.h;
    auto wgrid = [&](int params) { return grid_n(ctx, (int64_t)params * 32); };
    k_out_grad<<<grid_n(ctx, (int64_t)B * D.o), kThreads, 0, st>>>((int64_t)B * D.o, 1.0 / ((double)B * D.o), w.Y, T,
                                                                   w.dY);
    k_dense_bwd_w<<<wgrid(D.o * D.h + D.o), kThreads, 0, st>>>(B, D.h, D.o, w.dY, w.H2, gW3, gb3);
    k_dense_bwd_data<<<grid_n(ctx, (int64_t)B * D.h), kThreads, 0, st>>>(B, D.h, D.o, W3, w.dY, w.H2, w.dZ2);
    k_dense_bwd_w<<<wgrid(D.h * D.h + D.h), kThreads, 0, st>>>(B, D.h, D.h, w.dZ2, w.H1, gW2, gb2);
    k_dense_bwd_data<<<grid_n(ctx, (int64_t)B * D.h), kThreads, 0, st>>>(B, D.h, D.h, W2, w.dZ2, w.H1, w.dZ1);
    k_dense_bwd_w<<<wgrid(D.h * D.d + D.h), kThreads, 0, st>>>(B, D.d, D.h, w.dZ1, X, gW1, gb1);
}

int check_net(sscg_ctx* ctx, int d, int h, int o, int B) {
    if (d < 1 || h < 1 || o < 1 || d > 4096 || h > 4096 || o > 4096 || B < 1 || B > (1 << 22))
        return set_err(ctx, SSCG_ERR_INVALID, "network sizes d=%d h=%d o=%d or batch %d out of range", d, h, o, B);
    return SSCG_OK;
}

int check_ws(sscg_ctx* ctx, void* ws, size_t have, size_t need) {
    if (!ws || have < need || ((uintptr_t)ws & 255))
        return set_err(ctx, SSCG_ERR_SPACE, "workspace needs %zu bytes, 256-byte aligned (got %zu)", need, have);
    return SSCG_OK;
}

// ----------------------------------------------------------- features

constexpr int kFeatPart = 9;  // partial values per CTA, see k_features

__device__ __forceinline__ double feat_combine(int q, double x, double y) {
    return q == 2 || q == 8 ? fmin(x, y) : (q == 3 ? fmax(x, y) : x + y);
}

// Rows per thread summed in FP32 before the sums move into FP64.
constexpr int kFeatFlush = 8;

// One pass over the matrix.  Per row: ln d_i and (sum_{j!=i} |a_ij|) / d_i;
// per nonzero off-diagonal entry: ln c_ij with c_ij = |a_ij| / sqrt(d_i d_j).
// The features need about seven digits, so the pass reads the FP32 copies
// of the values and of 1/d and works in FP32 (GB300's FP64 rate is 1/57 of
// its FP32 rate); sums are taken about a shift (row 0's values) so that the
// second moments keep their digits, in FP32 over at most kFeatFlush rows and
// in FP64 beyond.  Partials per CTA: [sum ed, sum ed^2, min ld, max ld,
// sum dom, count, sum ec, sum ec^2, min lc] with ed = ld - shift_d,
// ec = lc - shift_c; the last CTA combines them in CTA order and writes the
// ten features.
__global__ void __launch_bounds__(kThreads) k_features(int n, const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col,
                                                       const float* __restrict__ vf,
                                                       const float* __restrict__ dinv_f, double* __restrict__ part,
                                                       double* __restrict__ feat, Ctrl* ctrl) {
    const float shift_d = -logf(dinv_f[0]);
    float shift_c = 0.f;
    for (int k = rowptr[0]; k < rowptr[1]; k++) {
        const int j = col[k];
        const float a = fabsf(vf[k]);
        if (j != 0 && a > 0.f) {
            shift_c = logf(a * sqrtf(dinv_f[0] * dinv_f[j]));
            break;
        }
    }
    double v[kFeatPart] = {0.0, 0.0, INFINITY, -INFINITY, 0.0, 0.0, 0.0, 0.0, INFINITY};
    float f_ed = 0.f, f_ed2 = 0.f, f_dom = 0.f, f_ec = 0.f, f_ec2 = 0.f;
    float ldmin = INFINITY, ldmax = -INFINITY, lcmin = INFINITY;
    int cnt = 0, rows = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float dfi = dinv_f[i];
        const float ld = -logf(dfi);
        const float ed = ld - shift_d;
        f_ed += ed;
        f_ed2 = fmaf(ed, ed, f_ed2);
        ldmin = fminf(ldmin, ld);
        ldmax = fmaxf(ldmax, ld);
        float off = 0.f;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            const int j = col[k];
            if (j == i) continue;
            const float a = fabsf(vf[k]);
            off += a;
            if (a > 0.f) {
                const float lc = logf(a * sqrtf(dfi * dinv_f[j]));
                const float ec = lc - shift_c;
                cnt++;
                f_ec += ec;
                f_ec2 = fmaf(ec, ec, f_ec2);
                lcmin = fminf(lcmin, lc);
            }
        }
        f_dom = fmaf(off, dfi, f_dom);
        if (++rows == kFeatFlush) {
            v[0] += f_ed;
            v[1] += f_ed2;
            v[4] += f_dom;
            v[6] += f_ec;
            v[7] += f_ec2;
            f_ed = f_ed2 = f_dom = f_ec = f_ec2 = 0.f;
            rows = 0;
        }
    }
    v[0] += f_ed;
    v[1] += f_ed2;
    v[2] = ldmin;
    v[3] = ldmax;
    v[4] += f_dom;
    v[5] = (double)cnt;
    v[6] += f_ec;
    v[7] += f_ec2;
    v[8] = lcmin;
    __shared__ double sh[kFeatPart][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kFeatPart; q++) {
        double t = v[q];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t = feat_combine(q, t, __shfl_xor_sync(0xffffffffu, t, m));
        if (lane == 0) sh[q][warp] = t;
    }
    __syncthreads();
    const int G = gridDim.x;
    if (threadIdx.x < kFeatPart) {
        const int q = threadIdx.x;
        double t = sh[q][0];
        for (int w = 1; w < nw; w++) t = feat_combine(q, t, sh[q][w]);
        part[(size_t)q * G + blockIdx.x] = t;
    }
    if (!last_cta(&ctrl->ticket[0])) return;
    // warp q combines partial q: lanes stride the CTAs, then a fixed shuffle tree
    __shared__ double a[kFeatPart];
    for (int q = warp; q < kFeatPart; q += nw) {
        double t = q == 2 || q == 8 ? INFINITY : (q == 3 ? -INFINITY : 0.0);
        for (int b = lane; b < G; b += 32) t = feat_combine(q, t, __ldcg(part + (size_t)q * G + b));
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t = feat_combine(q, t, __shfl_xor_sync(0xffffffffu, t, m));
        if (lane == 0) a[q] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double md = a[0] / n;  // mean of ed
        const double vd = fmax(a[1] / n - md * md, 0.0);
        const double cn = a[5];
        const double mc = cn > 0.0 ? a[6] / cn : 0.0;
        const double vc = cn > 0.0 ? fmax(a[7] / cn - mc * mc, 0.0) : 0.0;
        const double mean_d = (double)shift_d + md;
        feat[0] = log((double)n) / 3.0;
        feat[1] = log((double)rowptr[n] / (double)n);
        feat[2] = mean_d;
        feat[3] = sqrt(vd);
        feat[4] = a[2] - mean_d;
        feat[5] = a[3] - mean_d;
        feat[6] = a[4] / n;
        feat[7] = cn > 0.0 ? (double)shift_c + mc : 0.0;
        feat[8] = sqrt(vc);
        feat[9] = cn > 0.0 ? a[8] : 0.0;
    }
}

// Inference on one feature vector by one CTA (thread u computes hidden unit
// u).  The model blob is [x_mean (d), x_std (d), y_mean (o), y_std (o),
// theta]; x is normalised as (f - x_mean) / x_std and the outputs are
// de-normalised as y y_std + y_mean.  Writes exp of the first two outputs
// (lambda_min, lambda_max) into ctrl->scratch[0..1].
__global__ void __launch_bounds__(kThreads) k_mlp_bounds(int d, int h, int o, const double* __restrict__ model,
                                                         const double* __restrict__ feat, Ctrl* ctrl) {
    __shared__ double x[SSCG_NFEAT], h1[kThreads], h2[kThreads];
    const double* xm = model;
    const double* xs = xm + d;
    const double* ym = xs + d;
    const double* ys = ym + o;
    const double* W1 = ys + o;
    const double* b1 = W1 + (size_t)h * d;
    const double* W2 = b1 + h;
    const double* b2 = W2 + (size_t)h * h;
    const double* W3 = b2 + h;
    const double* b3 = W3 + (size_t)o * h;
    const int u = threadIdx.x;
    if (u < d) x[u] = (feat[u] - xm[u]) / xs[u];
    __syncthreads();
    if (u < h) {
        double t = b1[u];
        for (int k = 0; k < d; k++) t = fma(W1[(size_t)u * d + k], x[k], t);
        h1[u] = tanh(t);
    }
    __syncthreads();
    if (u < h) {
        double t = b2[u];
        for (int k = 0; k < h; k++) t = fma(W2[(size_t)u * h + k], h1[k], t);
        h2[u] = tanh(t);
    }
    __syncthreads();
    if (u < 2) {
        double t = b3[u];
        for (int k = 0; k < h; k++) t = fma(W3[(size_t)u * h + k], h2[k], t);
        ctrl->scratch[u] = exp(fma(t, ys[u], ym[u]));
    }
}

size_t features_ws_bytes() {
    Carve c(nullptr, 0);
    c.take<Ctrl>(1);
    c.take<double>((size_t)kFeatPart * kMaxGrid);
    c.take<double>(SSCG_NFEAT);
    return c.used;
}

// Launches k_features into ws; hands back the control block and the device
// address of the ten features.
int run_features(sscg_ctx* ctx, const sscg_mat* m, void* ws, Ctrl** ctrl_out, double** feat_out) {
    Carve c(ws, 0);
    Ctrl* ctrl = c.take<Ctrl>(1);
    double* part = c.take<double>((size_t)kFeatPart * kMaxGrid);
    double* feat = c.take<double>(SSCG_NFEAT);
    SSCG_CUDA(ctx, cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), ctx->stream));
    const int G = grid_for(ctx, m->n, 4);
    k_features<<<G, kThreads, 0, ctx->stream>>>((int)m->n, m->rowptr, m->col, m->vhi, m->dinv_f, part, feat, ctrl);
    SSCG_CUDA(ctx, cudaGetLastError());
    *ctrl_out = ctrl;
    *feat_out = feat;
    return SSCG_OK;
}

}  // namespace

size_t features_workspace() { return features_ws_bytes(); }

int bounds_mlp(sscg_ctx* ctx, const sscg_mat* m, int h, const double* model, void* ws, size_t ws_bytes, double* lmin,
               double* lmax) {
    if (!m || !model || !lmin || !lmax) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    if (h < 1 || h > kThreads) return set_err(ctx, SSCG_ERR_INVALID, "hidden width %d outside 1..%d", h, kThreads);
    if (int e = check_ws(ctx, ws, ws_bytes, features_ws_bytes())) return e;
    Ctrl* ctrl;
    double* f;
    if (int e = run_features(ctx, m, ws, &ctrl, &f)) return e;
    k_mlp_bounds<<<1, kThreads, 0, ctx->stream>>>(SSCG_NFEAT, h, 2, model, f, ctrl);
    SSCG_CUDA(ctx, cudaGetLastError());
    double out[2];
    SSCG_CUDA(ctx, cudaMemcpyAsync(out, ctrl->scratch, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
    SSCG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!(out[0] > 0.0) || !(out[1] > out[0]) || !std::isfinite(out[1]))
        return set_err(ctx, SSCG_ERR_NONFINITE, "network gave the interval [%g, %g]", out[0], out[1]);
    *lmin = out[0];
    *lmax = out[1];
    return SSCG_OK;
}

}  // namespace sscg

using namespace sscg;

extern "C" {

int64_t sscg_mlp_nparams(int d, int h, int o) {
    if (d < 1 || h < 1 || o < 1) return -1;
    return MlpDims{d, h, o}.np();
}

int sscg_mlp_workspace_bytes(int d, int h, int o, int batch, size_t* bytes) {
    if (!bytes || d < 1 || h < 1 || o < 1 || batch < 1) return SSCG_ERR_INVALID;
    *bytes = mlp_plan(MlpDims{d, h, o}, batch, nullptr).bytes;
    return SSCG_OK;
}

int sscg_mlp_forward(sscg_ctx* ctx, int d, int h, int o, const double* theta, int batch, const double* X, double* Y,
                     void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (int e = check_net(ctx, d, h, o, batch)) return e;
    if (!theta || !X || !Y) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    const MlpDims D{d, h, o};
    const MlpWork w = mlp_plan(D, batch, ws);
    if (int e = check_ws(ctx, ws, ws_bytes, w.bytes)) return e;
    launch_forward(ctx, D, theta, batch, X, w);
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaMemcpyAsync(Y, w.Y, sizeof(double) * (size_t)batch * o, cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    return SSCG_OK;
}

int sscg_mlp_loss_grad(sscg_ctx* ctx, int d, int h, int o, const double* theta, int batch, const double* X,
                       const double* T, double* grad, double* loss, void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (int e = check_net(ctx, d, h, o, batch)) return e;
    if (!theta || !X || !T || !grad) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    const MlpDims D{d, h, o};
    const MlpWork w = mlp_plan(D, batch, ws);
    if (int e = check_ws(ctx, ws, ws_bytes, w.bytes)) return e;
    launch_forward(ctx, D, theta, batch, X, w);
    launch_backward(ctx, D, theta, batch, X, T, w, grad);
    k_mse<<<1, kThreads, 0, ctx->stream>>>((int64_t)batch * o, w.Y, T, w.loss);
    SSCG_CUDA(ctx, cudaGetLastError());
    if (loss) {
        SSCG_CUDA(ctx, cudaMemcpyAsync(loss, w.loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        SSCG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return SSCG_OK;
}

int sscg_mlp_adam_step(sscg_ctx* ctx, int64_t np, double* theta, const double* grad, double* m, double* v, double lr,
                       double beta1, double beta2, double eps, int t) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (np < 1 || !theta || !grad || !m || !v || t < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
        !(beta2 >= 0.0 && beta2 < 1.0) || !(eps >= 0.0))
        return set_err(ctx, SSCG_ERR_INVALID, "bad Adam arguments");
    k_adam<<<grid_n(ctx, np), kThreads, 0, ctx->stream>>>(np, theta, grad, m, v, lr, beta1, beta2, eps,
                                                          1.0 - pow(beta1, (double)t), 1.0 - pow(beta2, (double)t));
    SSCG_CUDA(ctx, cudaGetLastError());
    return SSCG_OK;
}

int sscg_mlp_train(sscg_ctx* ctx, int d, int h, int o, double* theta, int batch, const double* X, const double* T,
                   int epochs, double lr, double* loss_hist, void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (int e = check_net(ctx, d, h, o, batch)) return e;
    if (!theta || !X || !T || epochs < 0 || !(lr > 0.0)) return set_err(ctx, SSCG_ERR_INVALID, "bad argument");
    const MlpDims D{d, h, o};
    const MlpWork w = mlp_plan(D, batch, ws);
    if (int e = check_ws(ctx, ws, ws_bytes, w.bytes)) return e;
    cudaStream_t st = ctx->stream;
    const int64_t np = D.np();
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    SSCG_CUDA(ctx, cudaMemsetAsync(w.m, 0, sizeof(double) * np, st));
    SSCG_CUDA(ctx, cudaMemsetAsync(w.v, 0, sizeof(double) * np, st));
    for (int t = 1; t <= epochs; t++) {
        launch_forward(ctx, D, theta, batch, X, w);
        launch_backward(ctx, D, theta, batch, X, T, w, w.grad);
        if (loss_hist) {
            k_mse<<<1, kThreads, 0, st>>>((int64_t)batch * o, w.Y, T, w.loss);
            SSCG_CUDA(ctx, cudaMemcpyAsync(loss_hist + (t - 1), w.loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        k_adam<<<grid_n(ctx, np), kThreads, 0, st>>>(np, theta, w.grad, w.m, w.v, lr, b1, b2, eps,
                                                     1.0 - pow(b1, (double)t), 1.0 - pow(b2, (double)t));
        if ((t & 63) == 0) SSCG_CUDA(ctx, cudaGetLastError());
    }
    SSCG_CUDA(ctx, cudaGetLastError());
    SSCG_CUDA(ctx, cudaStreamSynchronize(st));
    return SSCG_OK;
}

int sscg_features_workspace_bytes(size_t* bytes) {
    if (!bytes) return SSCG_ERR_INVALID;
    *bytes = features_ws_bytes();
    return SSCG_OK;
}

int sscg_mat_features(sscg_ctx* ctx, const sscg_mat* m, double* feat, void* ws, size_t ws_bytes) {
    if (!ctx) return SSCG_ERR_INVALID;
    if (!m || !feat) return set_err(ctx, SSCG_ERR_INVALID, "null argument");
    if (int e = check_ws(ctx, ws, ws_bytes, features_ws_bytes())) return e;
    Ctrl* ctrl;
    double* f;
    if (int e = run_features(ctx, m, ws, &ctrl, &f)) return e;
    SSCG_CUDA(ctx, cudaMemcpyAsync(feat, f, sizeof(double) * SSCG_NFEAT, cudaMemcpyDeviceToDevice, ctx->stream));
    return SSCG_OK;
}

int sscg_bounds_mlp(sscg_ctx* ctx, const sscg_mat* m, int h, const double* model, void* ws, size_t ws_bytes,
                    double* lmin, double* lmax) {
    if (!ctx) return SSCG_ERR_INVALID;
    return bounds_mlp(ctx, m, h, model, ws, ws_bytes, lmin, lmax);
}

int sscg_set_bounds_model(sscg_mat* m, int h, const double* model) {
    if (!m) return SSCG_ERR_INVALID;
    if (model && (h < 1 || h > kThreads)) return SSCG_ERR_INVALID;
    m->bounds_model = model;
    m->bounds_h = model ? h : 0;
    return SSCG_OK;
}

}  // extern "C"
