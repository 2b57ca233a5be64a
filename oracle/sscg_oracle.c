/*
 * Oracle for the preconditioned s-step CG method of arXiv 2501.03743.
 *
 * TEST INFRASTRUCTURE ONLY (see sscg_oracle.h).  Plain FP64 loops, written
 * to be checked against the paper by eye:
 *   - orc_pcg        : Algorithm 1 (PCG-HS)
 *   - orc_pfcg       : Algorithm 2 (PFCG-NN, Notay's flexible CG)
 *   - orc_pcgs       : Algorithm 3 with Algorithms 4 (pMPK), 5 (cvm), 6 (SW)
 *   - orc_pcgs_gram  : the same s-step method with the Gram blocks formed
 *                      directly from Section II-A's definitions
 *                      (W = P^T A P, beta from W_{i-1} beta + c = 0,
 *                      alpha from W alpha = m), for any polynomial basis
 *   - orc_lanczos_bounds : Ritz values from the CG coefficients
 *   - orc_mlp_*      : the spectral-bound network in FP64
 *   - orc_features   : matrix features the network reads
 *   - orc_adam_step  : the optimiser step that trains it
 * Compiled with -ffp-contract=off so that x86 and Arm hosts round the same.
 */
#include "sscg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_CHUNK 4096

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- basics */

double orc_dot(int64_t n, const double* a, const double* b) {
    int64_t nc = (n + ORC_CHUNK - 1) / ORC_CHUNK;
    if (nc == 0) return 0.0;
    double* part = (double*)malloc((size_t)nc * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; c++) {
        int64_t lo = c * ORC_CHUNK, hi = lo + ORC_CHUNK < n ? lo + ORC_CHUNK : n;
        double t = 0.0;
        for (int64_t i = lo; i < hi; i++) t += a[i] * b[i];
        part[c] = t;
    }
    double s = 0.0;
    for (int64_t c = 0; c < nc; c++) s += part[c];
    free(part);
    return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(orc_dot(n, a, a)); }

void orc_spmv(const orc_csr* A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; i++) {
        double t = 0.0;
        for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) t += A->val[k] * x[A->col[k]];
        y[i] = t;
    }
}

void orc_diag(const orc_csr* A, double* d) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; i++) {
        double t = 0.0;
        for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
            if (A->col[k] == i) t += A->val[k];
        d[i] = t;
    }
}

static double* vec(int64_t n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* ------------------------------------------------------- preconditioner */

/* z = B^-1 r.
 * NONE: z = r.  JACOBI: z = D^-1 r.
 * CHEB: `degree` steps of Chebyshev acceleration (Saad, Iterative Methods
 * for Sparse Linear Systems, Sec. 12.3) applied to D^-1 A y = D^-1 r from
 * y = 0, with theta, delta the centre and half-width of [lmin, lmax]:
 *   rho_0 = delta/theta, d_0 = g/theta, y_1 = d_0, res_1 = g - M d_0,
 *   rho_k = 1/(2 theta/delta - rho_{k-1}),
 *   d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) res_k,
 *   y_{k+1} = y_k + d_k, res_{k+1} = res_k - M d_k,   M = D^-1 A, g = D^-1 r.
 * The result is p(M) D^-1 r with 1 - lambda p(lambda) equal to
 * T_degree((theta - lambda)/delta) / T_degree(theta/delta). */
int orc_prec_apply(const orc_csr* A, const orc_prec* B, const double* r, double* z) {
    int64_t n = A->n;
    if (B == NULL || B->kind == ORC_PREC_NONE) {
        memcpy(z, r, (size_t)n * sizeof(double));
        return ORC_OK;
    }
    double* d = vec(n);
    orc_diag(A, d);
    if (B->kind == ORC_PREC_JACOBI) {
        for (int64_t i = 0; i < n; i++) z[i] = r[i] / d[i];
        free(d);
        return ORC_OK;
    }
    if (B->kind != ORC_PREC_CHEB || B->degree < 1 || !(B->lmax > B->lmin) || !(B->lmin >= 0.0)) {
        free(d);
        return ORC_ERR_INVALID;
    }
    double theta = 0.5 * (B->lmax + B->lmin), delta = 0.5 * (B->lmax - B->lmin);
    double* g = vec(n);
    double* dk = vec(n);
    double* res = vec(n);
    double* Md = vec(n);
    for (int64_t i = 0; i < n; i++) g[i] = r[i] / d[i];
    double rho = delta / theta;
    for (int64_t i = 0; i < n; i++) { dk[i] = g[i] / theta; z[i] = dk[i]; res[i] = g[i]; }
    for (int k = 1; k < B->degree; k++) {
        orc_spmv(A, dk, Md);
        for (int64_t i = 0; i < n; i++) res[i] -= Md[i] / d[i];
        double rho_new = 1.0 / (2.0 * theta / delta - rho);
        for (int64_t i = 0; i < n; i++) {
            dk[i] = rho_new * rho * dk[i] + (2.0 * rho_new / delta) * res[i];
            z[i] += dk[i];
        }
        rho = rho_new;
    }
    free(d); free(g); free(dk); free(res); free(Md);
    return ORC_OK;
}

/* ----------------------------------------------------- dense Cholesky */

/* Solve A X = B for SPD A (n x n, column-major) and nrhs right-hand sides
 * (n x nrhs, column-major) by the Cholesky factorisation A = L L^T.
 * Returns ORC_BREAKDOWN if a pivot is not positive or not finite. */
int orc_chol_solve(int n, const double* A, int nrhs, const double* B, double* X) {
    double* L = (double*)calloc((size_t)n * n, sizeof(double));
    for (int j = 0; j < n; j++) {
        double djj = A[j + (size_t)j * n];
        for (int k = 0; k < j; k++) djj -= L[j + (size_t)k * n] * L[j + (size_t)k * n];
        if (!(djj > 0.0) || !isfinite(djj)) { free(L); return ORC_BREAKDOWN; }
        double ljj = sqrt(djj);
        L[j + (size_t)j * n] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = A[i + (size_t)j * n];
            for (int k = 0; k < j; k++) t -= L[i + (size_t)k * n] * L[j + (size_t)k * n];
            L[i + (size_t)j * n] = t / ljj;
        }
    }
    for (int c = 0; c < nrhs; c++) {
        const double* b = B + (size_t)c * n;
        double* x = X + (size_t)c * n;
        for (int i = 0; i < n; i++) { /* L y = b */
            double t = b[i];
            for (int k = 0; k < i; k++) t -= L[i + (size_t)k * n] * x[k];
            x[i] = t / L[i + (size_t)i * n];
        }
        for (int i = n - 1; i >= 0; i--) { /* L^T x = y */
            double t = x[i];
            for (int k = i + 1; k < n; k++) t -= L[k + (size_t)i * n] * x[k];
            x[i] = t / L[i + (size_t)i * n];
        }
        for (int i = 0; i < n; i++)
            if (!isfinite(x[i])) { free(L); return ORC_BREAKDOWN; }
    }
    free(L);
    return ORC_OK;
}

/* --------------------------------------------------------- bookkeeping */

static void hist_push(orc_result* res, double v) {
    if (res && res->hist && res->hist_len < res->hist_cap) res->hist[res->hist_len] = v;
    if (res) res->hist_len++;
}

static void result_init(orc_result* res) {
    if (!res) return;
    res->status = ORC_NOT_CONVERGED;
    res->iters = 0;
    res->relres = NAN;
    res->hist_len = 0;
}

static int finish(orc_result* res, int status, int iters, double relres) {
    if (res) {
        res->status = status;
        res->iters = iters;
        res->relres = relres;
        if (res->hist_len > res->hist_cap) res->hist_len = res->hist_cap;
    }
    return status;
}

/* ------------------------------------------------------ Algorithm 1 */

/* PCG-HS (Algorithm 1).  Runs at most `maxit` iterations (k = 0..maxit-1);
 * stops when ||r_{k+1}||_2 / ||b||_2 < tol.  If cg_alpha / cg_beta are not
 * NULL they receive alpha_k and beta_k of every iteration (for Lanczos). */
int orc_pcg(const orc_csr* A, const orc_prec* B, const double* b, double* x,
            double tol, int maxit, orc_result* res, double* cg_alpha, double* cg_beta) {
    int64_t n = A->n;
    result_init(res);
    if (n <= 0 || maxit < 0) return finish(res, ORC_ERR_INVALID, 0, NAN);
    double* r = vec(n); double* u = vec(n); double* p = vec(n); double* sv = vec(n);
    double nb = nrm2(n, b);
    if (nb == 0.0) { memset(x, 0, (size_t)n * sizeof(double)); free(r); free(u); free(p); free(sv); hist_push(res, 0.0); return finish(res, ORC_OK, 0, 0.0); }
    orc_spmv(A, x, sv);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - sv[i];               /* r0 = b - A x0 */
    if (orc_prec_apply(A, B, r, u) != ORC_OK) { free(r); free(u); free(p); free(sv); return finish(res, ORC_ERR_INVALID, 0, NAN); }
    memcpy(p, u, (size_t)n * sizeof(double));                          /* p0 = u0 */
    double rho = orc_dot(n, u, r);
    double relres = nrm2(n, r) / nb;
    hist_push(res, relres);
    int status = ORC_NOT_CONVERGED, k;
    if (relres < tol) { status = ORC_OK; k = 0; goto done; }
    for (k = 0; k < maxit; k++) {
        orc_spmv(A, p, sv);                                            /* s_k = A p_k */
        double pts = orc_dot(n, p, sv);
        if (!(pts > 0.0) || !isfinite(pts) || !isfinite(rho)) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / pts;                                      /* alpha_k */
        for (int64_t i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * sv[i]; }
        orc_prec_apply(A, B, r, u);                                    /* u_{k+1} = B^-1 r_{k+1} */
        double rho_new = orc_dot(n, u, r);
        double beta = rho_new / rho;                                   /* beta_k */
        for (int64_t i = 0; i < n; i++) p[i] = u[i] + beta * p[i];     /* p_{k+1} */
        if (cg_alpha) cg_alpha[k] = alpha;
        if (cg_beta) cg_beta[k] = beta;
        rho = rho_new;
        relres = nrm2(n, r) / nb;
        hist_push(res, relres);
        if (!isfinite(relres)) { status = ORC_BREAKDOWN; k++; break; }
        if (relres < tol) { status = ORC_OK; k++; break; }
    }
done:
    free(r); free(u); free(p); free(sv);
    return finish(res, status, k, relres);
}

/* ------------------------------------------------------ Algorithm 2 */

/* PFCG-NN (Algorithm 2), with the final return taken as x_{k+1}. */
int orc_pfcg(const orc_csr* A, const orc_prec* B, const double* b, double* x,
             double tol, int maxit, orc_result* res) {
    int64_t n = A->n;
    result_init(res);
    if (n <= 0 || maxit < 0) return finish(res, ORC_ERR_INVALID, 0, NAN);
    double* r = vec(n); double* u = vec(n); double* p = vec(n); double* s = vec(n); double* w = vec(n);
    double nb = nrm2(n, b);
    if (nb == 0.0) { memset(x, 0, (size_t)n * sizeof(double)); free(r); free(u); free(p); free(s); free(w); hist_push(res, 0.0); return finish(res, ORC_OK, 0, 0.0); }
    orc_spmv(A, x, w);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - w[i];
    double relres = nrm2(n, r) / nb;
    hist_push(res, relres);
    int status = ORC_NOT_CONVERGED, k = 0;
    if (relres < tol) { status = ORC_OK; goto done; }
    orc_prec_apply(A, B, r, u);
    memcpy(p, u, (size_t)n * sizeof(double));
    orc_spmv(A, u, w);
    memcpy(s, w, (size_t)n * sizeof(double));
    double alpha = orc_dot(n, u, r);
    double rho = orc_dot(n, p, s);
    if (!(rho > 0.0)) { status = ORC_BREAKDOWN; goto done; }
    for (int64_t i = 0; i < n; i++) { x[i] += alpha / rho * p[i]; r[i] -= alpha / rho * s[i]; }
    relres = nrm2(n, r) / nb;
    hist_push(res, relres);
    k = 1;
    if (relres < tol) { status = ORC_OK; goto done; }
    for (; k < maxit; k++) {
        orc_prec_apply(A, B, r, u);
        orc_spmv(A, u, w);
        double ak = orc_dot(n, u, r), bk = orc_dot(n, u, w), gk = orc_dot(n, u, s);
        double rho_new = bk - gk * gk / rho;
        if (!(rho_new > 0.0) || !isfinite(rho_new)) { status = ORC_BREAKDOWN; break; }
        double c = gk / rho;
        for (int64_t i = 0; i < n; i++) {
            p[i] = u[i] - c * p[i];
            s[i] = w[i] - c * s[i];
        }
        rho = rho_new;
        for (int64_t i = 0; i < n; i++) { x[i] += ak / rho * p[i]; r[i] -= ak / rho * s[i]; }
        relres = nrm2(n, r) / nb;
        hist_push(res, relres);
        if (relres < tol) { status = ORC_OK; k++; break; }
    }
done:
    free(r); free(u); free(p); free(s); free(w);
    return finish(res, status, k, relres);
}

/* ------------------------------------------- Algorithms 3, 4, 5 and 6 */

/* Column j (0-based) of an n x m column-major block. */
#define COL(P, n, j) ((P) + (size_t)(j) * (size_t)(n))

/* pMPK (Algorithm 4): P(:,1) = B^-1 x, then alternately A and B^-1, with
 * the pin/pout bookkeeping that leaves U = P(:,1:s) and A U = P(:,s+1:2s). */
static int pmpk(const orc_csr* A, const orc_prec* B, const double* x, int s, double* P) {
    int64_t n = A->n;
    if (orc_prec_apply(A, B, x, COL(P, n, 0)) != ORC_OK) return ORC_ERR_INVALID;
    int pin = 1, pout = s + 1; /* 1-based, as in the listing */
    for (int j = 2; j <= 2 * s; j++) {
        if (j % 2 == 0)
            orc_spmv(A, COL(P, n, pin - 1), COL(P, n, pout - 1));
        else
            orc_prec_apply(A, B, COL(P, n, pin - 1), COL(P, n, pout - 1));
        int ptemp = pin;
        pin = pout;
        pout = ptemp + 1;
    }
    return ORC_OK;
}

/* cvm (Algorithm 5): vm(1:s) = P(:,1:s)^T r, vm(s+1:2s) = P(:,1:s)^T P(:,2s). */
static void cvm(int64_t n, const double* P, const double* r, int s, double* vm) {
    for (int j = 0; j < s; j++) vm[j] = orc_dot(n, COL(P, n, j), r);
    for (int j = 0; j < s; j++) vm[s + j] = orc_dot(n, COL(P, n, j), COL(P, n, 2 * s - 1));
}

/* SW (Algorithm 6), 1-based indices kept in the comments.
 *   rhs(s-1+i) = -( vm(i) + sum_{j<i} rhs(s-1+j) alpha(s-i+j) ) / alpha(s)
 *   b1(i,j)    = -rhs(i+j-1)        for all i, j in 1..s
 *   W_old beta = b1;   W = Hankel(vm) - b1 beta;   W alpha = vm(1:s)
 * The b1 loop runs over every j: the listing's "j = 1:i-1" bound would
 * leave b1 strictly lower triangular, while b1 = -c_i, the Hankel matrix of
 * r_i^T (B^-1 A)^(l+j-1) z_{i-1} (Section II-A), is full and symmetric.
 * On entry alpha and W hold the previous step's values. */
static int sw(int s, const double* vm, double* alpha, double* beta, double* W, double* b1_out) {
    double* rhs = (double*)calloc((size_t)(2 * s - 1), sizeof(double));
    double* b1 = (double*)calloc((size_t)s * s, sizeof(double));
    double* H = (double*)calloc((size_t)s * s, sizeof(double));
    double* tmp = (double*)calloc((size_t)s * s, sizeof(double));
    int st = ORC_OK;
    double as = alpha[s - 1];
    if (as == 0.0 || !isfinite(as)) { st = ORC_BREAKDOWN; goto out; }
    for (int i = 1; i <= s; i++) {
        double t = vm[i - 1];
        for (int j = 1; j <= i - 1; j++) t += rhs[s - 1 + j - 1] * alpha[s - i + j - 1];
        rhs[s - 1 + i - 1] = -t / as;
    }
    for (int i = 1; i <= s; i++)
        for (int j = 1; j <= s; j++) b1[(i - 1) + (size_t)(j - 1) * s] = -rhs[i + j - 1 - 1];
    if (b1_out) memcpy(b1_out, b1, sizeof(double) * s * s);
    st = orc_chol_solve(s, W, s, b1, beta);                       /* W_old beta = b1 */
    if (st != ORC_OK) goto out;
    for (int i = 1; i <= s; i++)
        for (int j = 1; j <= s; j++) H[(i - 1) + (size_t)(j - 1) * s] = vm[i + j - 1];
    for (int i = 0; i < s; i++)                                    /* W = H - b1 beta */
        for (int j = 0; j < s; j++) {
            double t = H[i + (size_t)j * s];
            for (int k = 0; k < s; k++) t -= b1[i + (size_t)k * s] * beta[k + (size_t)j * s];
            tmp[i + (size_t)j * s] = t;
        }
    memcpy(W, tmp, sizeof(double) * s * s);
    st = orc_chol_solve(s, W, 1, vm, alpha);                       /* W alpha = vm(1:s) */
out:
    free(rhs); free(b1); free(H); free(tmp);
    return st;
}

/* Block updates of Algorithm 3:
 *   Pnew(:,1:s)    += Pold(:,1:s) beta;      x += Pnew(:,1:s) alpha
 *   Pnew(:,s+1:2s) += Pold(:,s+1:2s) beta;   r -= Pnew(:,s+1:2s) alpha */
static void block_update(int64_t n, int s, double* Pnew, const double* Pold, const double* beta,
                         const double* alpha, double* x, double* r) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        for (int half = 0; half < 2; half++) {
            double newv[64];
            for (int j = 0; j < s; j++) {
                double t = Pnew[i + (size_t)(half * s + j) * n];
                for (int l = 0; l < s; l++) t += Pold[i + (size_t)(half * s + l) * n] * beta[l + (size_t)j * s];
                newv[j] = t;
            }
            double acc = 0.0;
            for (int j = 0; j < s; j++) {
                Pnew[i + (size_t)(half * s + j) * n] = newv[j];
                acc += newv[j] * alpha[j];
            }
            if (half == 0) x[i] += acc; else r[i] -= acc;
        }
    }
}

static void trace_step(orc_trace* tr, int64_t n, int s, int step, const double* U, const double* AU,
                       const double* P, const double* AP, const double* r, const double* x,
                       const double* W, const double* alpha, const double* beta,
                       const double* b1, const double* vm) {
    if (!tr || step >= tr->cap) return;
    size_t ns = (size_t)n * s, ss = (size_t)s * s;
    if (tr->U && U) memcpy(tr->U + step * ns, U, ns * sizeof(double));
    if (tr->AU && AU) memcpy(tr->AU + step * ns, AU, ns * sizeof(double));
    if (tr->P && P) memcpy(tr->P + step * ns, P, ns * sizeof(double));
    if (tr->AP && AP) memcpy(tr->AP + step * ns, AP, ns * sizeof(double));
    if (tr->r) memcpy(tr->r + step * (size_t)n, r, (size_t)n * sizeof(double));
    if (tr->x) memcpy(tr->x + step * (size_t)n, x, (size_t)n * sizeof(double));
    if (tr->W) memcpy(tr->W + step * ss, W, ss * sizeof(double));
    if (tr->alpha) memcpy(tr->alpha + step * (size_t)s, alpha, (size_t)s * sizeof(double));
    if (tr->beta) memcpy(tr->beta + step * ss, beta, ss * sizeof(double));
    if (tr->b1 && b1) memcpy(tr->b1 + step * ss, b1, ss * sizeof(double));
    if (tr->vm && vm) memcpy(tr->vm + step * (size_t)(2 * s), vm, (size_t)(2 * s) * sizeof(double));
    tr->len = step + 1;
}

/* PCGs (Algorithm 3) with pMPK, cvm and SW exactly as listed (monomial
 * basis).  `maxit` bounds the outer steps k = 0..maxit-1.  The two blocks
 * P1, P2 of the listing alternate between "new" (even k: P2, odd k: P1)
 * and "old"; P1 starts at zero.  Stops when ||r||_2/||b||_2 < tol. */
int orc_pcgs(const orc_csr* A, const orc_prec* B, const double* b, double* x,
             int s, double tol, int maxit, orc_result* res, orc_trace* tr) {
    int64_t n = A->n;
    result_init(res);
    if (n <= 0 || s < 1 || s > 32 || maxit < 0) return finish(res, ORC_ERR_INVALID, 0, NAN);
    if (tr) tr->len = 0;
    size_t blk = (size_t)n * 2 * s;
    double* P1 = (double*)calloc(blk, sizeof(double));
    double* P2 = (double*)calloc(blk, sizeof(double));
    double* U = (double*)calloc(blk, sizeof(double));
    double* r = vec(n);
    double* vm = (double*)calloc((size_t)2 * s, sizeof(double));
    double* W = (double*)calloc((size_t)s * s, sizeof(double));
    double* alpha = (double*)calloc((size_t)s, sizeof(double));
    double* beta = (double*)calloc((size_t)s * s, sizeof(double));
    double* b1 = (double*)calloc((size_t)s * s, sizeof(double));
    int status = ORC_NOT_CONVERGED, k = 0;
    double relres = NAN;
    double nb = nrm2(n, b);
    if (nb == 0.0) { memset(x, 0, (size_t)n * sizeof(double)); relres = 0.0; hist_push(res, 0.0); status = ORC_OK; goto done; }
    orc_spmv(A, x, r);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];                 /* r = b - A x0 */
    relres = nrm2(n, r) / nb;
    hist_push(res, relres);
    if (relres < tol) { status = ORC_OK; goto done; }
    for (k = 0; k < maxit; k++) {
        double* Pnew = (k % 2 == 0) ? P2 : P1;
        double* Pold = (k % 2 == 0) ? P1 : P2;
        if (pmpk(A, B, r, s, Pnew) != ORC_OK) { status = ORC_ERR_INVALID; break; }
        if (tr) memcpy(U, Pnew, blk * sizeof(double));
        cvm(n, Pnew, r, s, vm);
        int st;
        if (k == 0) {
            for (int i = 1; i <= s; i++)
                for (int j = 1; j <= s; j++) W[(i - 1) + (size_t)(j - 1) * s] = vm[i + j - 1];
            memset(beta, 0, sizeof(double) * s * s);
            memset(b1, 0, sizeof(double) * s * s);
            st = orc_chol_solve(s, W, 1, vm, alpha);
        } else {
            st = sw(s, vm, alpha, beta, W, b1);
        }
        if (st != ORC_OK) { status = ORC_BREAKDOWN; break; }
        block_update(n, s, Pnew, Pold, beta, alpha, x, r);
        relres = nrm2(n, r) / nb;
        hist_push(res, relres);
        trace_step(tr, n, s, k, U, U + (size_t)n * s, Pnew, Pnew + (size_t)n * s, r, x, W, alpha, beta, b1, vm);
        if (!isfinite(relres)) { status = ORC_BREAKDOWN; k++; break; }
        if (relres < tol) { status = ORC_OK; k++; break; }
    }
done:
    free(P1); free(P2); free(U); free(r); free(vm); free(W); free(alpha); free(beta); free(b1);
    return finish(res, status, k, relres);
}

/* Basis block of the direct-Gram variant: u_1 = B^-1 r, AU_j = A u_j and
 *   monomial : u_{j+1} = B^-1 A u_j                                (Alg. 4)
 *   Chebyshev: u_2 = (B^-1 A u_1 - c u_1)/delta,
 *              u_{j+1} = 2 (B^-1 A u_j - c u_j)/delta - u_{j-1},
 * with c, delta the centre and half-width of [blo, bhi], bounds of the
 * spectrum of B^-1 A (the scaled Chebyshev basis named in Section IV). */
int orc_newton_shifts(int s, double lo, double hi, double* theta, double* sigma) {
    if (s < 1 || !(hi > lo)) return ORC_ERR_INVALID;
    const int m = s - 1;
    const double c = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    const double pi = 3.14159265358979323846;
    double* t = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int* used = (int*)calloc((size_t)(m > 0 ? m : 1), sizeof(int));
    for (int k = 0; k < m; k++) t[k] = c + delta * cos((2.0 * k + 1.0) * pi / (2.0 * m));
    for (int q = 0; q < m; q++) {
        int best = -1;
        double bv = -1.0;
        for (int k = 0; k < m; k++) {
            if (used[k]) continue;
            double v;
            if (q == 0) {
                v = fabs(t[k]);
            } else {
                v = 1.0;
                for (int i = 0; i < q; i++) v *= fabs(t[k] - theta[i]);
            }
            if (best < 0 || v > bv * (1.0 + 1e-12)) {  /* near-ties go to the lower index */
                bv = v;
                best = k;
            }
        }
        used[best] = 1;
        theta[q] = t[best];
    }
    *sigma = 0.25 * (hi - lo);
    free(t);
    free(used);
    return ORC_OK;
}

static int basis_block(const orc_csr* A, const orc_prec* B, const double* r, int s, int basis,
                       double blo, double bhi, double* U, double* AU, double* w) {
    int64_t n = A->n;
    double c = 0.5 * (bhi + blo), delta = 0.5 * (bhi - blo);
    double theta[32], sigma = 1.0;
    if (basis == ORC_BASIS_NEWTON && orc_newton_shifts(s, blo, bhi, theta, &sigma) != ORC_OK) return ORC_ERR_INVALID;
    if (orc_prec_apply(A, B, r, COL(U, n, 0)) != ORC_OK) return ORC_ERR_INVALID;
    for (int j = 0; j < s; j++) {
        orc_spmv(A, COL(U, n, j), COL(AU, n, j));
        if (j + 1 == s) break;
        orc_prec_apply(A, B, COL(AU, n, j), w);
        double* un = COL(U, n, j + 1);
        const double* uj = COL(U, n, j);
        if (basis == ORC_BASIS_MONOMIAL) {
            memcpy(un, w, (size_t)n * sizeof(double));
        } else if (basis == ORC_BASIS_NEWTON) {  /* u_{j+1} = (B^-1 A u_j - theta_j u_j) / sigma */
            for (int64_t i = 0; i < n; i++) un[i] = (w[i] - theta[j] * uj[i]) / sigma;
        } else if (j == 0) {
            for (int64_t i = 0; i < n; i++) un[i] = (w[i] - c * uj[i]) / delta;
        } else {
            const double* um = COL(U, n, j - 1);
            for (int64_t i = 0; i < n; i++) un[i] = 2.0 * (w[i] - c * uj[i]) / delta - um[i];
        }
    }
    return ORC_OK;
}

/* The s-step method with Gram blocks formed directly (Section II-A):
 *   G = U^T (A U)           (lower triangle, i >= j: u_i . (A u_j))
 *   m = U^T r
 *   k = 0: W = G, beta = 0
 *   k > 0: C = (A P_old)^T U, W_old beta = -C, W = G + C^T beta
 *   W alpha = m;  P = U + P_old beta;  AP = AU + AP_old beta;
 *   x += P alpha;  r -= AP alpha.
 * W = G + C^T beta is P^T A P once P_old^T A P = 0 is imposed, and
 * m = P^T r because r is orthogonal to P_old. */
int orc_pcgs_gram(const orc_csr* A, const orc_prec* B, const double* b, double* x,
                  int s, int basis, double blo, double bhi, double tol, int maxit,
                  orc_result* res, orc_trace* tr) {
    int64_t n = A->n;
    result_init(res);
    if (n <= 0 || s < 1 || s > 32 || maxit < 0) return finish(res, ORC_ERR_INVALID, 0, NAN);
    if (basis != ORC_BASIS_MONOMIAL && !(bhi > blo)) return finish(res, ORC_ERR_INVALID, 0, NAN);
    if (tr) tr->len = 0;
    size_t ns = (size_t)n * s;
    double* U = (double*)calloc(ns, sizeof(double));
    double* AU = (double*)calloc(ns, sizeof(double));
    double* P = (double*)calloc(ns, sizeof(double));
    double* AP = (double*)calloc(ns, sizeof(double));
    double* Po = (double*)calloc(ns, sizeof(double));
    double* APo = (double*)calloc(ns, sizeof(double));
    double* r = vec(n); double* w = vec(n);
    double* G = (double*)calloc((size_t)s * s, sizeof(double));
    double* C = (double*)calloc((size_t)s * s, sizeof(double));
    double* W = (double*)calloc((size_t)s * s, sizeof(double));
    double* m = (double*)calloc((size_t)s, sizeof(double));
    double* alpha = (double*)calloc((size_t)s, sizeof(double));
    double* beta = (double*)calloc((size_t)s * s, sizeof(double));
    int status = ORC_NOT_CONVERGED, k = 0;
    double relres = NAN;
    double nb = nrm2(n, b);
    if (nb == 0.0) { memset(x, 0, (size_t)n * sizeof(double)); relres = 0.0; hist_push(res, 0.0); status = ORC_OK; goto done; }
    orc_spmv(A, x, r);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];
    relres = nrm2(n, r) / nb;
    hist_push(res, relres);
    if (relres < tol) { status = ORC_OK; goto done; }
    for (k = 0; k < maxit; k++) {
        if (basis_block(A, B, r, s, basis, blo, bhi, U, AU, w) != ORC_OK) { status = ORC_ERR_INVALID; break; }
        for (int i = 0; i < s; i++) {
            m[i] = orc_dot(n, COL(U, n, i), r);
            for (int j = 0; j <= i; j++) {
                G[i + (size_t)j * s] = orc_dot(n, COL(U, n, i), COL(AU, n, j));
                G[j + (size_t)i * s] = G[i + (size_t)j * s];
            }
        }
        int st = ORC_OK;
        if (k == 0) {
            memcpy(W, G, sizeof(double) * s * s);
            memset(beta, 0, sizeof(double) * s * s);
        } else {
            for (int l = 0; l < s; l++)
                for (int j = 0; j < s; j++) C[l + (size_t)j * s] = -orc_dot(n, COL(APo, n, l), COL(U, n, j));
            st = orc_chol_solve(s, W, s, C, beta);                 /* W_old beta = -C */
            if (st == ORC_OK) {
                for (int i = 0; i < s; i++)                         /* W = G + C^T beta */
                    for (int j = 0; j < s; j++) {
                        double t = G[i + (size_t)j * s];
                        for (int l = 0; l < s; l++) t -= C[l + (size_t)i * s] * beta[l + (size_t)j * s];
                        W[i + (size_t)j * s] = t;
                    }
            }
        }
        if (st == ORC_OK) st = orc_chol_solve(s, W, 1, m, alpha);
        if (st != ORC_OK) { status = ORC_BREAKDOWN; break; }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double xa = 0.0, ra = 0.0;
            for (int j = 0; j < s; j++) {
                double p = U[i + (size_t)j * n], ap = AU[i + (size_t)j * n];
                for (int l = 0; l < s; l++) {
                    p += Po[i + (size_t)l * n] * beta[l + (size_t)j * s];
                    ap += APo[i + (size_t)l * n] * beta[l + (size_t)j * s];
                }
                P[i + (size_t)j * n] = p;
                AP[i + (size_t)j * n] = ap;
                xa += p * alpha[j];
                ra += ap * alpha[j];
            }
            x[i] += xa;
            r[i] -= ra;
        }
        relres = nrm2(n, r) / nb;
        hist_push(res, relres);
        trace_step(tr, n, s, k, U, AU, P, AP, r, x, W, alpha, beta, NULL, NULL);
        double* t1 = Po; Po = P; P = t1;
        double* t2 = APo; APo = AP; AP = t2;
        if (!isfinite(relres)) { status = ORC_BREAKDOWN; k++; break; }
        if (relres < tol) { status = ORC_OK; k++; break; }
    }
done:
    free(U); free(AU); free(P); free(AP); free(Po); free(APo); free(r); free(w);
    free(G); free(C); free(W); free(m); free(alpha); free(beta);
    return finish(res, status, k, relres);
}

/* ------------------------------------------------- Lanczos / Ritz values */

/* Number of eigenvalues of the symmetric tridiagonal T (diagonal d[0..k-1],
 * off-diagonal e[0..k-2]) that are smaller than x: Sturm sequence count. */
static int sturm_count(int k, const double* d, const double* e, double x) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0.0) cnt++;
    for (int i = 1; i < k; i++) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

/* Smallest and largest eigenvalue of T by bisection on the Sturm count,
 * starting from the Gershgorin interval. */
int orc_tridiag_eig_extremes(int k, const double* d, const double* e, double* lo, double* hi) {
    if (k < 1) return ORC_ERR_INVALID;
    double a = d[0], b = d[0];
    for (int i = 0; i < k; i++) {
        double rad = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < k ? fabs(e[i]) : 0.0);
        if (d[i] - rad < a) a = d[i] - rad;
        if (d[i] + rad > b) b = d[i] + rad;
    }
    double span = b - a + 1e-300;
    a -= 1e-12 * span; b += 1e-12 * span;
    for (int which = 0; which < 2; which++) {
        int target = which == 0 ? 1 : k; /* eigenvalue index (1-based) */
        double l = a, h = b;
        for (int it = 0; it < 200 && h - l > 1e-15 * (fabs(l) + fabs(h)); it++) {
            double mid = 0.5 * (l + h);
            if (sturm_count(k, d, e, mid) >= target) h = mid; else l = mid;
        }
        if (which == 0) *lo = 0.5 * (l + h); else *hi = 0.5 * (l + h);
    }
    return ORC_OK;
}

/* Ritz values of B^-1 A from k steps of PCG on A y = r0 (y0 = 0): the
 * Lanczos tridiagonal built from the CG coefficients,
 *   T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T_{j,j+1} = sqrt(beta_j)/alpha_j
 * (Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.7.3). */
int orc_lanczos_bounds(const orc_csr* A, const orc_prec* B, const double* r0, int k,
                       double* lo, double* hi) {
    int64_t n = A->n;
    if (k < 1) return ORC_ERR_INVALID;
    double* a = (double*)calloc((size_t)k, sizeof(double));
    double* bb = (double*)calloc((size_t)k, sizeof(double));
    double* y = vec(n);
    orc_result res = {0};
    /* stop at an invariant Krylov space (to working precision): beyond it the
     * coefficients only carry rounding noise */
    orc_pcg(A, B, r0, y, 1e-14, k, &res, a, bb);
    int kk = res.iters;
    if (kk < 1) { free(a); free(bb); free(y); return ORC_BREAKDOWN; }
    double* d = (double*)calloc((size_t)kk, sizeof(double));
    double* e = (double*)calloc((size_t)kk, sizeof(double));
    for (int j = 0; j < kk; j++) {
        d[j] = 1.0 / a[j] + (j > 0 ? bb[j - 1] / a[j - 1] : 0.0);
        if (j + 1 < kk) e[j] = sqrt(bb[j]) / a[j];
    }
    int st = orc_tridiag_eig_extremes(kk, d, e, lo, hi);
    free(a); free(bb); free(y); free(d); free(e);
    return st;
}

/* -------------------------------------------------------------- MLP */

int64_t orc_mlp_nparams(int d, int h, int o) {
    return (int64_t)h * d + h + (int64_t)h * h + h + (int64_t)o * h + o;
}

/* Forward pass for one sample; h1, h2 receive the hidden activations. */
static void mlp_sample(int d, int h, int o, const double* th, const double* x,
                       double* h1, double* h2, double* y) {
    const double* W1 = th; const double* b1 = W1 + (size_t)h * d;
    const double* W2 = b1 + h; const double* b2 = W2 + (size_t)h * h;
    const double* W3 = b2 + h; const double* b3 = W3 + (size_t)o * h;
    for (int i = 0; i < h; i++) {
        double t = b1[i];
        for (int j = 0; j < d; j++) t += W1[(size_t)i * d + j] * x[j];
        h1[i] = tanh(t);
    }
    for (int i = 0; i < h; i++) {
        double t = b2[i];
        for (int j = 0; j < h; j++) t += W2[(size_t)i * h + j] * h1[j];
        h2[i] = tanh(t);
    }
    for (int i = 0; i < o; i++) {
        double t = b3[i];
        for (int j = 0; j < h; j++) t += W3[(size_t)i * h + j] * h2[j];
        y[i] = t;
    }
}

void orc_mlp_forward(int d, int h, int o, const double* theta, int batch, const double* X, double* Y) {
    double* h1 = (double*)malloc(sizeof(double) * h);
    double* h2 = (double*)malloc(sizeof(double) * h);
    for (int b = 0; b < batch; b++) mlp_sample(d, h, o, theta, X + (size_t)b * d, h1, h2, Y + (size_t)b * o);
    free(h1); free(h2);
}

/* Mean squared error L = 1/(batch*o) sum (Y - T)^2 and its gradient with
 * respect to every parameter (reverse-mode chain rule, tanh' = 1 - tanh^2). */
double orc_mlp_loss_grad(int d, int h, int o, const double* th, int batch, const double* X,
                         const double* T, double* grad) {
    int64_t np = orc_mlp_nparams(d, h, o);
    memset(grad, 0, sizeof(double) * (size_t)np);
    const double* W2 = th + (size_t)h * d + h;
    const double* W3 = W2 + (size_t)h * h + h;
    double* gW1 = grad; double* gb1 = gW1 + (size_t)h * d;
    double* gW2 = gb1 + h; double* gb2 = gW2 + (size_t)h * h;
    double* gW3 = gb2 + h; double* gb3 = gW3 + (size_t)o * h;
    double* h1 = (double*)malloc(sizeof(double) * h);
    double* h2 = (double*)malloc(sizeof(double) * h);
    double* y = (double*)malloc(sizeof(double) * o);
    double* dy = (double*)malloc(sizeof(double) * o);
    double* d2 = (double*)malloc(sizeof(double) * h);
    double* d1 = (double*)malloc(sizeof(double) * h);
    double loss = 0.0, scale = 1.0 / ((double)batch * o);
    for (int b = 0; b < batch; b++) {
        const double* x = X + (size_t)b * d;
        mlp_sample(d, h, o, th, x, h1, h2, y);
        for (int i = 0; i < o; i++) {
            double e = y[i] - T[(size_t)b * o + i];
            loss += e * e * scale;
            dy[i] = 2.0 * e * scale;
        }
        for (int i = 0; i < o; i++) {
            gb3[i] += dy[i];
            for (int j = 0; j < h; j++) gW3[(size_t)i * h + j] += dy[i] * h2[j];
        }
        for (int j = 0; j < h; j++) {
            double t = 0.0;
            for (int i = 0; i < o; i++) t += W3[(size_t)i * h + j] * dy[i];
            d2[j] = t * (1.0 - h2[j] * h2[j]);
        }
        for (int i = 0; i < h; i++) {
            gb2[i] += d2[i];
            for (int j = 0; j < h; j++) gW2[(size_t)i * h + j] += d2[i] * h1[j];
        }
        for (int j = 0; j < h; j++) {
            double t = 0.0;
            for (int i = 0; i < h; i++) t += W2[(size_t)i * h + j] * d2[i];
            d1[j] = t * (1.0 - h1[j] * h1[j]);
        }
        for (int i = 0; i < h; i++) {
            gb1[i] += d1[i];
            for (int j = 0; j < d; j++) gW1[(size_t)i * d + j] += d1[i] * x[j];
        }
    }
    free(h1); free(h2); free(y); free(dy); free(d2); free(d1);
    return loss;
}

/* ------------------------------------------------- features and optimiser */

int orc_features(const orc_csr* A, double* f) {
    int64_t n = A->n;
    double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_diag(A, d);
    /* first pass: means, extremes, dominance */
    double s1 = 0.0, dmin = INFINITY, dmax = -INFINITY, dom = 0.0;
    double cnt = 0.0, c1 = 0.0, cmin = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        if (!(d[i] > 0.0)) { free(d); return -1; }
        double ld = log(d[i]);
        s1 += ld;
        if (ld < dmin) dmin = ld;
        if (ld > dmax) dmax = ld;
    }
    for (int64_t i = 0; i < n; i++) {
        double off = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
            int64_t j = A->col[k];
            if (j == i) continue;
            double a = fabs(A->val[k]);
            off += a;
            if (a > 0.0) {
                double lc = log(a / sqrt(d[i] * d[j]));
                cnt += 1.0; c1 += lc;
                if (lc < cmin) cmin = lc;
            }
        }
        dom += off / d[i];
    }
    double mean = s1 / (double)n, cm = cnt > 0.0 ? c1 / cnt : 0.0;
    /* second pass: spreads about the means */
    double s2 = 0.0, c2 = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double e = log(d[i]) - mean;
        s2 += e * e;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
            int64_t j = A->col[k];
            double a = fabs(A->val[k]);
            if (j == i || !(a > 0.0)) continue;
            double ec = log(a / sqrt(d[i] * d[j])) - cm;
            c2 += ec * ec;
        }
    }
    f[0] = log((double)n) / 3.0;
    f[1] = log((double)A->rowptr[n] / (double)n);
    f[2] = mean;
    f[3] = sqrt(s2 / (double)n);
    f[4] = dmin - mean;
    f[5] = dmax - mean;
    f[6] = dom / (double)n;
    f[7] = cm;
    f[8] = cnt > 0.0 ? sqrt(c2 / cnt) : 0.0;
    f[9] = cnt > 0.0 ? cmin : 0.0;
    free(d);
    return 0;
}

void orc_adam_step(int64_t np, double* theta, const double* g, double* m, double* v,
                   double lr, double b1, double b2, double eps, int t) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < np; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
