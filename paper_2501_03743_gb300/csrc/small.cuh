// The s x s coefficient solves of the s-step method, done on chip in FP64
// by one warp (Section III moves them to the host; here they run in the
// last CTA of the kernel that completes the Gram/moment reduction).
#pragma once

#include "common.cuh"

namespace sscg {

// In-place Cholesky A = L L^T of an s x s column-major matrix in shared
// memory (lower triangle overwritten by L), lanes parallel over rows, with
// rinv[k] = 1 / L_kk: one reciprocal square root per pivot, the column below
// it scaled by that reciprocal (a multiplication, where a division would sit
// on the serial chain).  Returns false (in every lane) if a pivot is not
// positive or not finite.
__device__ __forceinline__ bool warp_cholesky(double* A, int s, double* rinv) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < s; k++) {
        __syncwarp();
        double d = A[k + k * s];
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double r = rsqrt(d);
        __syncwarp();
        if (lane == 0) {
            A[k + k * s] = d * r;
            rinv[k] = r;
        }
        if (lane > k && lane < s) A[lane + k * s] *= r;
        __syncwarp();
        if (lane > k && lane < s) {
            double lik = A[lane + k * s];
            for (int j = k + 1; j <= lane; j++) A[lane + j * s] -= lik * A[j + k * s];
        }
    }
    __syncwarp();
    return true;
}

// Solve L L^T X = B for `nrhs` column-major right-hand sides (in place),
// lanes parallel over columns, multiplying by rinv[i] = 1 / L_ii (from
// warp_cholesky) rather than dividing.  Returns false if a result is not finite.
__device__ __forceinline__ bool warp_chol_solve(const double* L, int s, double* B, int nrhs, const double* rinv) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    for (int c = lane; c < nrhs; c += 32) {
        double* b = B + c * s;
        for (int i = 0; i < s; i++) {
            double t = b[i];
            for (int k = 0; k < i; k++) t -= L[i + k * s] * b[k];
            b[i] = t * rinv[i];
        }
        for (int i = s - 1; i >= 0; i--) {
            double t = b[i];
            for (int k = i + 1; k < s; k++) t -= L[k + i * s] * b[k];
            b[i] = t * rinv[i];
            ok = ok && isfinite(b[i]);
        }
    }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
}

// Scratch for the solves: 4 s x s matrices and 3 vectors, for s <= MS, and
// shared-memory copies of the inputs the monomial step reads more than once
// (the moments mu_0..mu_{2s-1} and the previous alpha).
template <int MS>
struct SmallScratchT {
    double L[MS * MS];
    double X[MS * MS];
    double Wn[MS * MS];
    double b1[MS * MS];
    double a[MS];
    double c[MS];
    double mu[2 * MS];
    double al[MS];
    double r[MS];  // reciprocals of the Cholesky factor's diagonal
};
using SmallScratch = SmallScratchT<kMaxS>;

// Algorithm 6 (SW) for the monomial basis, or its first-step form, by one
// warp.  Inputs in ctrl: mu[0..2s-1] (vm(k) = mu_{k-1}), and for step > 0
// the previous alpha and the Cholesky factor of the previous W (Wl, Wr: each
// step keeps the factor it formed for its own W, so W_prev is not factored
// again).  Outputs: W, its factor, alpha, beta.  Returns an sscg_status (0 or
// SSCG_BREAKDOWN).
//   step 0:  W(a,b) = mu_{a+b+1}, beta = 0, W alpha = (mu_0..mu_{s-1})
//   step >0: c_t = -(mu_t + sum_{j<t} c_j alpha_prev(s-1-t+j)) / alpha_prev(s-1)
//            b1(a,b) = -c_{a+b+1-s} (zero when a+b+1 < s), all a, b
//            W_prev beta = b1;  W = H - b1 beta;  W alpha = m
// (0-based indices; b1 filled over all (a, b), the consistent reading of
// Algorithm 6, whose b1 equals -c_i of Section II-A.)
template <class SC>
__device__ inline int warp_sw_monomial(Ctrl* ctrl, int s, int step, SC* sc) {
    const int lane = threadIdx.x & 31;
    // the moments and the previous alpha copied to shared memory by the whole
    // warp at once: the serial steps below then read no global memory
    for (int e = lane; e < 2 * s; e += 32) sc->mu[e] = ctrl->mu[e];
    if (step > 0)
        for (int e = lane; e < s; e += 32) sc->al[e] = ctrl->alpha[e];
    __syncwarp();
    const double* mu = sc->mu;
    if (step == 0) {
        for (int e = lane; e < s * s; e += 32) {
            int a = e % s, b = e / s;
            sc->Wn[e] = mu[a + b + 1];
            sc->L[e] = mu[a + b + 1];
            sc->X[e] = 0.0;
        }
        if (lane < s) sc->a[lane] = mu[lane];
        __syncwarp();
        if (!warp_cholesky(sc->L, s, sc->r)) return 2;
        if (!warp_chol_solve(sc->L, s, sc->a, 1, sc->r)) return 2;
    } else {
        const double* al = sc->al;
        double as = al[s - 1];
        if (as == 0.0 || !isfinite(as)) return 2;
        if (lane == 0) {
            const double ias = 1.0 / as;
            for (int t = 0; t < s; t++) {
                double v = mu[t];
                for (int j = 0; j < t; j++) v += sc->c[j] * al[s - 1 - t + j];
                sc->c[t] = -v * ias;
            }
        }
        __syncwarp();
        for (int e = lane; e < s * s; e += 32) {
            int a = e % s, b = e / s;
            int q = a + b + 1 - s;
            double v = q >= 0 ? -sc->c[q] : 0.0;
            sc->b1[e] = v;
            sc->X[e] = v;
            sc->L[e] = ctrl->Wl[e];  // the factor of W_prev, from the previous step
        }
        if (lane < s) sc->r[lane] = ctrl->Wr[lane];
        __syncwarp();
        if (!warp_chol_solve(sc->L, s, sc->X, s, sc->r)) return 2;  // beta = W_prev^-1 b1
        for (int e = lane; e < s * s; e += 32) {
            int a = e % s, b = e / s;
            double t = mu[a + b + 1];
            for (int k = 0; k < s; k++) t -= sc->b1[a + k * s] * sc->X[k + b * s];
            sc->Wn[e] = t;
        }
        __syncwarp();
        for (int e = lane; e < s * s; e += 32) sc->L[e] = sc->Wn[e];
        if (lane < s) sc->a[lane] = mu[lane];
        __syncwarp();
        if (!warp_cholesky(sc->L, s, sc->r)) return 2;
        if (!warp_chol_solve(sc->L, s, sc->a, 1, sc->r)) return 2;
    }
    for (int e = lane; e < s * s; e += 32) {
        ctrl->W[e] = sc->Wn[e];
        ctrl->Wl[e] = sc->L[e];
        ctrl->beta[e] = sc->X[e];
    }
    if (lane < s) {
        ctrl->Wr[lane] = sc->r[lane];
        ctrl->alpha[lane] = sc->a[lane];
    }
    __syncwarp();
    return 0;
}

// The same step with Gram blocks formed directly (any basis):
//   step 0:  W = G, beta = 0;  step > 0: W_prev beta = -C, W = G + C^T beta
//   W alpha = m (+ beta^T q when q = P_old^T r was formed: the right-hand
//   side P^T r of Section II-A for a residual that is not exactly orthogonal
//   to P_old, as after residual replacement).
//   G, C (column-major, C(l,j) = (A p_l^old) . u_j), m and q in ctrl; for
//   step > 0 the Cholesky factor of W_prev that the previous step kept (Wl, Wr).
__device__ inline int warp_sw_gram(Ctrl* ctrl, int s, int step, SmallScratch* sc) {
    const int lane = threadIdx.x & 31;
    if (step == 0) {
        for (int e = lane; e < s * s; e += 32) {
            sc->Wn[e] = ctrl->G[e];
            sc->X[e] = 0.0;
        }
    } else {
        for (int e = lane; e < s * s; e += 32) {
            sc->L[e] = ctrl->Wl[e];  // the factor of W_prev, from the previous step
            sc->X[e] = -ctrl->C[e];
        }
        if (lane < s) sc->r[lane] = ctrl->Wr[lane];
        __syncwarp();
        if (!warp_chol_solve(sc->L, s, sc->X, s, sc->r)) return 2;
        for (int e = lane; e < s * s; e += 32) {
            int i = e % s, j = e / s;
            double t = ctrl->G[e];
            for (int l = 0; l < s; l++) t += ctrl->C[l + i * s] * sc->X[l + j * s];
            sc->Wn[e] = t;
        }
    }
    __syncwarp();
    for (int e = lane; e < s * s; e += 32) sc->L[e] = sc->Wn[e];
    if (lane < s) {
        double mi = ctrl->m[lane];
        if (step > 0 && ctrl->with_q)
            for (int l = 0; l < s; l++) mi += sc->X[l + lane * s] * ctrl->q[l];
        sc->a[lane] = mi;
    }
    __syncwarp();
    if (!warp_cholesky(sc->L, s, sc->r)) return 2;
    if (!warp_chol_solve(sc->L, s, sc->a, 1, sc->r)) return 2;
    for (int e = lane; e < s * s; e += 32) {
        ctrl->W[e] = sc->Wn[e];
        ctrl->Wl[e] = sc->L[e];
        ctrl->beta[e] = sc->X[e];
    }
    if (lane < s) {
        ctrl->Wr[lane] = sc->r[lane];
        ctrl->alpha[lane] = sc->a[lane];
    }
    __syncwarp();
    return 0;
}

}  // namespace sscg
