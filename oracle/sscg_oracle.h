/*
 * Oracle for the preconditioned s-step Conjugate Gradient method
 * (Chronopoulos and Gear, as summarised in "Communication-reduced Conjugate
 * Gradient Variants for GPU-accelerated Clusters", arXiv 2501.03743).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, serial-in-spirit FP64 CPU
 * restatement of the paper's algorithms, used to check the CUDA library.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA
 * path; the only thing both sides share is the seeded input generator,
 * which holds none of the method's arithmetic.
 *
 * Conventions: CSR with int32 row pointers and column indices, FP64 values.
 * All vectors are FP64 host arrays owned by the caller.  Every reduction
 * is summed in fixed 4096-element chunks, so results do not depend on the
 * number of OpenMP threads.
 */
#ifndef SSCG_ORACLE_H
#define SSCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PREC_NONE = 0, ORC_PREC_JACOBI = 1, ORC_PREC_CHEB = 2 };
enum { ORC_BASIS_MONOMIAL = 0, ORC_BASIS_CHEBYSHEV = 1, ORC_BASIS_NEWTON = 2 };
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_BREAKDOWN = 2, ORC_ERR_INVALID = -1 };

typedef struct {
    int64_t n;
    const int32_t* rowptr; /* n+1 entries */
    const int32_t* col;    /* rowptr[n] entries */
    const double* val;     /* rowptr[n] entries */
} orc_csr;

/* Preconditioner B.  JACOBI: B = diag(A).  CHEB: B^-1 = p(D^-1 A) D^-1 with
 * p from `degree` steps of Chebyshev acceleration over [lmin, lmax], the
 * spectral interval of D^-1 A (degree 1 is Jacobi scaled by 2/(lmin+lmax)). */
typedef struct {
    int kind;
    int degree;
    double lmin, lmax;
} orc_prec;

typedef struct {
    int status;      /* ORC_OK / ORC_NOT_CONVERGED / ORC_BREAKDOWN */
    int iters;       /* PCG: iterations; s-step: outer steps */
    double relres;   /* recursive ||r||_2 / ||b||_2 at exit */
    double* hist;    /* caller-owned, may be NULL: relres before step 1, then after each step */
    int hist_cap;
    int hist_len;
} orc_result;

/* Optional per-outer-step record of the s-step internals, for invariant
 * checks on tiny systems.  Each pointer may be NULL; arrays are indexed
 * [step][...] with room for `cap` steps.  Blocks are column-major n x s. */
typedef struct {
    int cap;
    double* U;      /* cap * n * s   : basis block before the beta update   */
    double* AU;     /* cap * n * s   : A times the basis block              */
    double* P;      /* cap * n * s   : search directions after the update   */
    double* AP;     /* cap * n * s                                           */
    double* r;      /* cap * n       : residual after the step              */
    double* x;      /* cap * n       : iterate after the step               */
    double* W;      /* cap * s * s   : column-major                         */
    double* alpha;  /* cap * s                                              */
    double* beta;   /* cap * s * s   : column-major                         */
    double* b1;     /* cap * s * s   : SW right-hand side (literal variant) */
    double* vm;     /* cap * 2s      : moments (literal variant)            */
    int len;
} orc_trace;

void orc_spmv(const orc_csr* A, const double* x, double* y);
double orc_dot(int64_t n, const double* a, const double* b);
void orc_diag(const orc_csr* A, double* d);
int orc_prec_apply(const orc_csr* A, const orc_prec* B, const double* r, double* z);

int orc_pcg(const orc_csr* A, const orc_prec* B, const double* b, double* x,
            double tol, int maxit, orc_result* res, double* cg_alpha, double* cg_beta);

int orc_pcgs(const orc_csr* A, const orc_prec* B, const double* b, double* x,
             int s, double tol, int maxit, orc_result* res, orc_trace* tr);

/* basis: ORC_BASIS_MONOMIAL, ORC_BASIS_CHEBYSHEV (three-term recurrence over
 * [blo, bhi]) or ORC_BASIS_NEWTON (orc_newton_shifts over [blo, bhi]). */
int orc_pcgs_gram(const orc_csr* A, const orc_prec* B, const double* b, double* x,
                  int s, int basis, double blo, double bhi, double tol, int maxit,
                  orc_result* res, orc_trace* tr);

/* Shifts of the Newton basis over the interval [lo, hi] of B^-1 A (Section IV
 * names the Newton basis; the shifts are this project's reading): the s - 1
 * zeros of the Chebyshev polynomial T_{s-1} mapped to [lo, hi],
 * t_k = c + delta cos((2k + 1) pi / (2 (s - 1))), put in Leja order (first
 * the point of largest modulus, then each next point maximising the product
 * of its distances to the points already chosen; scores within 1e-12
 * relative of each other count as ties and go to the lower index k),
 * and the scale sigma = (hi - lo) / 4, the logarithmic capacity of the
 * interval.  The basis is u_1 = B^-1 r, u_{j+1} = (B^-1 A u_j - theta_j u_j)
 * / sigma.  Returns ORC_ERR_INVALID for s < 1 or an empty interval. */
int orc_newton_shifts(int s, double lo, double hi, double* theta, double* sigma);

int orc_pfcg(const orc_csr* A, const orc_prec* B, const double* b, double* x,
             double tol, int maxit, orc_result* res);

int orc_chol_solve(int n, const double* A, int nrhs, const double* B, double* X);

int orc_tridiag_eig_extremes(int k, const double* d, const double* e, double* lo, double* hi);
/* Extreme Ritz values of B^-1 A from at most k CG-Lanczos steps from r0;
 * CG stops early once ||r|| <= 1e-14 ||r0|| (the Krylov space is then
 * invariant to working precision). */
int orc_lanczos_bounds(const orc_csr* A, const orc_prec* B, const double* r0, int k,
                       double* lo, double* hi);

/* Spectral-bound MLP, FP64: x -> tanh(W1 x + b1) -> tanh(W2 h + b2) -> W3 h + b3.
 * Parameters packed as [W1 (h x d, row-major), b1 (h), W2 (h x h), b2 (h),
 * W3 (o x h), b3 (o)].  X is batch x d row-major, Y batch x o. */
int64_t orc_mlp_nparams(int d, int h, int o);
void orc_mlp_forward(int d, int h, int o, const double* theta, int batch, const double* X, double* Y);
double orc_mlp_loss_grad(int d, int h, int o, const double* theta, int batch, const double* X,
                         const double* T, double* grad);

/* Matrix features for the spectral-bound network (the paper gives none; the
 * definitions are this project's).  With d_i = a_ii and, over the
 * off-diagonal entries, c_ij = |a_ij| / sqrt(d_i d_j):
 *   f0 = ln(n)/3            f1 = ln(nnz/n)
 *   f2 = mean ln d          f3 = std ln d (population)
 *   f4 = min ln d - f2      f5 = max ln d - f2
 *   f6 = mean_i (sum_{j!=i} |a_ij|) / d_i
 *   f7 = mean ln c          f8 = std ln c           f9 = min ln c
 * Off-diagonal zeros are skipped in f7-f9.  Returns 0, or -1 if a diagonal
 * entry is not positive. */
#define ORC_NFEAT 10
int orc_features(const orc_csr* A, double* f);

/* One Adam step (Kingma and Ba, 2015) with bias correction at step t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void orc_adam_step(int64_t np, double* theta, const double* g, double* m, double* v,
                   double lr, double b1, double b2, double eps, int t);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
