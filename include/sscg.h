/*
 * sscg - preconditioned s-step Conjugate Gradient (Chronopoulos and Gear) on
 * one NVIDIA GB300 (sm_103a), after "Communication-reduced Conjugate Gradient
 * Variants for GPU-accelerated Clusters" (Bernaschi, Carrozzo, Celestini,
 * Piperno, D'Ambra; arXiv 2501.03743).
 *
 * Plain C ABI: host or device pointers and sizes, no C++ or framework types.
 *
 * Memory.  The library never allocates device memory.  The caller provides
 *   - matrix storage (sscg_mat_storage_bytes), filled by sscg_mat_create_csr
 *     with a private copy of the CSR arrays plus derived data, and
 *   - solve workspace (sscg_solve_workspace_bytes / sscg_pcg_workspace_bytes).
 * Both must be device memory, 256-byte aligned, and stay alive and untouched
 * while a matrix handle or a solve uses them.  Workspace contents do not
 * carry over between calls.
 *
 * Streams.  Every device operation is issued on the stream given to
 * sscg_create (0 = legacy default stream).  Entry points that return host
 * results (solve info, bounds) synchronise that stream before returning.
 *
 * Errors.  Every entry point returns an sscg_status.  Negative values are
 * caller or CUDA errors: outputs are not written, and sscg_last_error gives
 * a one-line reason.  Positive values are numerical outcomes of a solve:
 * x holds the last iterate that passed every check and info is filled.
 *
 * Threads.  A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SSCG_H
#define SSCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSCG_OK = 0,
    SSCG_NOT_CONVERGED = 1, /* maxit outer steps without reaching tol (Alg. 3, last line) */
    SSCG_BREAKDOWN = 2,     /* singular or indefinite s x s system, alpha_s = 0, or a non-finite value */
    SSCG_TIMEOUT = 3,       /* a bounded on-device wait gave up */
    SSCG_ERR_INVALID = -1,  /* bad argument, size or option */
    SSCG_ERR_NOT_SPD = -2,  /* matrix rejected: a diagonal entry is not positive */
    SSCG_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    SSCG_ERR_SPACE = -4,    /* storage or workspace too small or misaligned */
    SSCG_ERR_NONFINITE = -5 /* NaN or Inf in the matrix values or right-hand side */
} sscg_status;

/* Polynomial basis of the s-step block (Section II-A uses the monomial basis;
 * Section IV names Newton and Chebyshev bases as the stable alternatives).
 * Both take the interval [basis_lmin, basis_lmax] of B^-1 A (estimated when
 * 0, 0).  CHEBYSHEV: the three-term recurrence of the Chebyshev polynomials
 * of the interval.  NEWTON: u_{j+1} = (B^-1 A u_j - theta_j u_j) / sigma with
 * the shifts theta_j the s - 1 Chebyshev points of the interval (zeros of
 * T_{s-1}) in Leja order and sigma = (basis_lmax - basis_lmin) / 4. */
typedef enum { SSCG_BASIS_MONOMIAL = 0, SSCG_BASIS_CHEBYSHEV = 1, SSCG_BASIS_NEWTON = 2 } sscg_basis;

/* Preconditioner B (Section II-A leaves B general: any SPD operator). */
typedef enum {
    SSCG_PREC_NONE = 0,   /* B = I */
    SSCG_PREC_JACOBI = 1, /* B = diag(A) */
    SSCG_PREC_CHEB = 2    /* B^-1 = p(D^-1 A) D^-1, Chebyshev polynomial over [lmin, lmax] */
} sscg_prec;

/* Arithmetic of the hot path.  F64 (the default, the paper's precision)
 * stores every value in FP64.  Where a GB300's scarce FP64 units would bound
 * a kernel, short sums and dot products run in 64-bit fixed point on the
 * integer units and are rounded once to FP64: the neighbour sums of stencil
 * rows, and with the monomial basis at s <= 6 the block update's P and Q
 * columns (P_j = U_j + sum_l P_old_l beta_lj; the row's values and the
 * column's coefficients aligned to their largest exponents with 8 guard bits:
 * error at most (1 + 7K/16) 2^-56 max|value| max|coefficient| for K terms,
 * plus half an ulp; SSCG_FMA_UPDATE selects FP64 FMAs there).  DF64 carries every basis, block and vector element as an
 * unevaluated sum of two FP32 numbers (about 48 significant bits, FP32
 * exponent range: right-hand sides and matrix values must lie well inside it)
 * and computes with the FP32 units, whose GB300 throughput is about 60 times
 * the FP64 rate; with the monomial basis it takes s <= 6 (larger s amplify its
 * rounding past 1e-7 of the FP64 solution).  MIXED stores the basis blocks and
 * matrix values in FP32 and accumulates the Gram sums, x and r in FP64, with
 * the true residual recomputed in FP64 every `replace_every` outer steps.  The
 * s x s solves are always FP64. */
typedef enum { SSCG_ARITH_F64 = 0, SSCG_ARITH_DF64 = 1, SSCG_ARITH_MIXED = 2 } sscg_arith;

/* Flags of sscg_opts.flags and sscg_mat_create_csr. */
#define SSCG_HOST_VECTORS 0x1u /* b and x are host pointers; copies happen inside the call */
#define SSCG_PROFILE 0x2u      /* bracket every kernel with CUDA events; fills the t_* fields of sscg_info */
#define SSCG_DIRECT_GRAM 0x4u  /* form the Gram blocks directly even for the monomial basis */
#define SSCG_FUSED_MPK 0x8u    /* several matrix-powers levels per launch, intermediate levels kept in L2 */
#define SSCG_ADAPTIVE_S 0x20u  /* after a breakdown restart from the last good iterate with s halved */
#define SSCG_FMA_UPDATE 0x40u  /* F64, s <= 6: form the block update's P and Q with FP64 FMAs, not fixed point */
#define SSCG_HOST_ARRAYS 0x1u  /* CSR arrays are host pointers (sscg_mat_create_csr) */
#define SSCG_MAT_CSR_ONLY 0x2u /* keep CSR kernels even for a constant-coefficient diagonal pattern */

/* Storage forms a matrix is multiplied in (sscg_mat_props.format).  CSR is
 * always kept; a matrix whose rows all hold entries on at most 32 fixed
 * offsets (j - i), each offset with one FP32-exact value, and a positive
 * constant diagonal (the constant-coefficient 7- and 27-point stencils) is
 * also stored as one 32-bit presence mask per row plus the offsets and their
 * values.  The s-step solver (monomial basis, Jacobi or no preconditioner)
 * and plain PCG with a diagonal preconditioner then read no column indices,
 * values or 1/diag; other solves use CSR. */
enum sscg_format { SSCG_FORMAT_CSR = 0, SSCG_FORMAT_DIA_CONST = 1 };

typedef struct sscg_ctx sscg_ctx;
typedef struct sscg_mat sscg_mat;

typedef struct {
    int s;              /* block size, 1..16 (Alg. 3) */
    int basis;          /* sscg_basis */
    double basis_lmin;  /* Chebyshev / Newton basis: spectral interval of B^-1 A; 0,0 = estimated by the solve:
                           the matrix's bounds network (sscg_set_bounds_model) under the Jacobi
                           preconditioner, else 20 Lanczos steps; widened by 0.95 / 1.05 */
    double basis_lmax;
    double tol;         /* stop when ||r||_2 / ||b||_2 < tol, r the recursive residual */
    int maxit;          /* outer steps (each is s CG steps), >= 0 */
    int arith;          /* sscg_arith */
    int replace_every;  /* MIXED: true-residual replacement period in outer steps (0 = 1) */
    unsigned flags;     /* SSCG_HOST_VECTORS */
} sscg_opts;

typedef struct {
    int status;                /* same value as returned */
    int outer_iters;           /* outer steps taken (PCG: iterations) */
    int64_t equiv_iters;       /* s * outer_iters: CG steps of solution improvement */
    double rel_res_recursive;  /* ||r||_2 / ||b||_2 of the recursive residual at exit */
    double rel_res_true;       /* ||b - A x||_2 / ||b||_2 recomputed at exit */
    double* hist;              /* caller-owned host array or NULL: rel. residual before step 1, then per step */
    int hist_cap;              /* entries available in hist */
    int hist_len;              /* entries written */
    int64_t kernel_launches;   /* kernels this call launched, including no-op launches queued past convergence */
    /* With SSCG_PROFILE: device time summed over the launches of the steps
     * actually taken, per kernel family, and the number of those launches.
     * s-step: mpk = matrix-powers levels (with the fused moments and, on the
     * last level, the s x s solves), update = block updates.  PCG: mpk =
     * SpMV + p.Ap, update = x, r update + dots, dir = direction update. */
    double t_init_ms, t_mpk_ms, t_update_ms, t_dir_ms, t_final_ms;
    int64_t n_mpk, n_update, n_dir;
    int s_final;               /* sscg_solve: the block size of the last segment (SSCG_ADAPTIVE_S halves it
                                  after each breakdown; otherwise opts->s) */
} sscg_info;

typedef struct {
    int64_t n, nnz;
    int64_t bandwidth;      /* max |i - j| over stored entries */
    int values_exact_fp32;  /* every value is exactly representable in FP32 */
    int max_row_nnz;
    double diag_min, diag_max;
    int prec, prec_degree;
    double prec_lmin, prec_lmax;
    int format;       /* sscg_format used by the s-step and PCG kernels */
    int dia_offsets;  /* offsets of the diagonal form (0 for CSR) */
} sscg_mat_props;

/* ------------------------------------------------------------ context */

/* Create a context bound to `cuda_stream` (a cudaStream_t, may be NULL).
 * Host memory only.  Errors: SSCG_ERR_INVALID (out == NULL),
 * SSCG_ERR_CUDA (no device or unsupported architecture). */
int sscg_create(sscg_ctx** out, void* cuda_stream);
int sscg_destroy(sscg_ctx* ctx);
const char* sscg_last_error(const sscg_ctx* ctx);
const char* sscg_status_str(int status);
/* Library version as major*10000 + minor*100 + patch. */
int sscg_version(void);

/* ------------------------------------------------------------- matrix */

/* Bytes of device storage sscg_mat_create_csr needs for an n x n matrix
 * with nnz stored entries (0 < n < 2^31, 0 <= nnz < 2^31). */
int sscg_mat_storage_bytes(int64_t n, int64_t nnz, size_t* bytes);

/* Create an SPD matrix from CSR arrays (Section III: row-block CSR; here one
 * block holds every row).  rowptr: n+1 int32, nondecreasing, rowptr[0] = 0,
 * rowptr[n] = nnz; colind: nnz int32 in [0, n); val: nnz FP64.  Arrays are
 * device pointers, or host pointers with SSCG_HOST_ARRAYS.  They are copied
 * into `storage` (device, >= sscg_mat_storage_bytes, 256-byte aligned) and
 * may be freed on return; `storage` is owned by the caller and must outlive
 * the handle.  Symmetry is the caller's promise and is not checked.
 * Errors: SSCG_ERR_INVALID (sizes, rowptr, colind out of range),
 * SSCG_ERR_NOT_SPD (a diagonal entry <= 0 or missing), SSCG_ERR_NONFINITE,
 * SSCG_ERR_SPACE, SSCG_ERR_CUDA.  Synchronises the context's stream. */
int sscg_mat_create_csr(sscg_ctx* ctx, int64_t n, int64_t nnz, const int32_t* rowptr,
                        const int32_t* colind, const double* val, unsigned flags,
                        void* storage, size_t storage_bytes, sscg_mat** out);
int sscg_mat_destroy(sscg_mat* mat); /* frees the host handle only */
int sscg_mat_props_get(const sscg_mat* mat, sscg_mat_props* props);

/* Select the preconditioner B used by every later solve with `mat`.
 * JACOBI ignores the other arguments.  CHEB: `degree` >= 1 steps of
 * Chebyshev acceleration on D^-1 A over [lmin, lmax] (0 < lmin < lmax), so
 * each apply costs degree-1 SpMVs; lmax must bound the spectrum of D^-1 A from
 * above for B to stay SPD.  Host-only.  Errors: SSCG_ERR_INVALID. */
int sscg_set_preconditioner(sscg_mat* mat, int prec, int degree, double lmin, double lmax);

/* ------------------------------------------------------------- solves */

/* Workspace bytes for sscg_solve with these options (depends on n, s, arith,
 * maxit and the SSCG_HOST_VECTORS flag). */
int sscg_solve_workspace_bytes(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);

/* Solve A x = b by the preconditioned s-step CG method (Algorithm 3 with the
 * matrix-powers kernel of Algorithm 4, the moments of Algorithm 5 and the
 * s x s solves of Algorithm 6 for the monomial basis; Gram blocks formed
 * directly for the Chebyshev basis).  b: n FP64; x: n FP64, x0 on entry and
 * the solution on exit (device pointers unless SSCG_HOST_VECTORS).
 * info may be NULL.  Returns SSCG_OK, SSCG_NOT_CONVERGED, SSCG_BREAKDOWN,
 * SSCG_TIMEOUT or a negative error (SSCG_ERR_INVALID also for DF64 with the
 * monomial basis and s > 6).  On b = 0, x = 0 and SSCG_OK.
 * With SSCG_ADAPTIVE_S in opts->flags, a breakdown restarts the solve from
 * the last good iterate with s halved (the budget stays maxit * s CG steps),
 * down to s = 1; info then sums the segments (s_final: the last one's s). */
int sscg_solve(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x,
               const sscg_opts* opts, sscg_info* info, void* workspace, size_t workspace_bytes);

/* Plain preconditioned CG (Algorithm 1) on the same kernels, the comparator
 * of the s-step method.  opts->s, basis are ignored; maxit counts iterations. */
int sscg_pcg_workspace_bytes(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);
int sscg_pcg_solve(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x,
                   const sscg_opts* opts, sscg_info* info, void* workspace, size_t workspace_bytes);

/* PFCG-NN (Algorithm 2): Notay's flexible preconditioned CG, the paper's
 * comparison solver.  Per iteration: one SpMV, one preconditioner apply, the
 * three coupled dot products alpha = u.r, beta = u.w, gamma = u.s in one
 * global reduction (with ||r||^2, so the stop test needs no second one) and
 * the two coupled axpy pairs p, s and x, r.  B: Jacobi or none (otherwise
 * SSCG_ERR_INVALID).  opts->s and basis are ignored; maxit counts iterations;
 * f64 or df64 arithmetic.  Vectors, workspace rules and returns as for
 * sscg_pcg_solve; SSCG_BREAKDOWN when rho_k = beta_k - gamma_k^2/rho_{k-1}
 * is not positive. */
int sscg_pfcg_workspace_bytes(const sscg_mat* mat, const sscg_opts* opts, size_t* bytes);
int sscg_pfcg_solve(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x,
                    const sscg_opts* opts, sscg_info* info, void* workspace, size_t workspace_bytes);

/* y = A x (device FP64 vectors of length n), the library's CSR SpMV. */
int sscg_spmv(sscg_ctx* ctx, const sscg_mat* mat, const double* x, double* y);

/* ---------------------------------------- solve with no allocation at all
 *
 * Some callers cannot allocate device memory: code that runs inside another
 * runtime's memory arena, plugins and embedded hosts that forbid cudaMalloc,
 * and services that must not allocate on the request path (an allocation can
 * synchronise the device or fail under memory pressure).  For them,
 * sscg_solve_static runs the same s-step solve as sscg_solve but takes its
 * workspace from a fixed array of SSCG_STATIC_SCRATCH_BYTES (16 MiB) that the
 * library itself places in device memory; every GPU that loads the library
 * holds that array until the process exits.  The caller still passes the
 * matrix, b and x.  The paper has no counterpart: this is a deployment
 * convenience, not part of the method.
 *
 * - Solves whose sscg_solve_workspace_bytes exceeds the array are rejected
 *   with SSCG_ERR_SPACE (about n <= 100,000 at s = 4).
 * - The call makes no cudaMalloc, cudaFree or other device allocation.
 * - The first call on each device looks the array's device address up
 *   (cudaGetSymbolAddress) with that device current, and caches it: make that
 *   first call before any stream capture.  The context's device must be the
 *   current device (SSCG_ERR_INVALID otherwise).
 * - All calls on a device share the one array, which keeps the last call's
 *   contents; the solve initialises everything it reads.  Calls whose work
 *   overlaps on the GPU (other streams or host threads) race on the array:
 *   serialise them.
 * - A device reset (cudaDeviceReset) reloads the library's device code and
 *   may move the array: the cached address is then stale.  Do not call
 *   sscg_solve_static on a device after resetting it in the same process.
 */
#define SSCG_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
int sscg_solve_static(sscg_ctx* ctx, const sscg_mat* mat, const double* b, double* x,
                      const sscg_opts* opts, sscg_info* info);

/* The Newton basis's shifts theta_0 .. theta_{s-2} and scale sigma over
 * [lmin, lmax], as the solver uses them (see sscg_basis).  Host-only.
 * Errors: SSCG_ERR_INVALID (s outside 1..16, an empty interval, null
 * outputs). */
int sscg_newton_shifts(int s, double lmin, double lmax, double* theta, double* sigma);

/* -------------------------------------------------- spectral bounds */

/* Workspace bytes for sscg_estimate_bounds with `steps` Lanczos steps. */
int sscg_bounds_workspace_bytes(const sscg_mat* mat, int steps, size_t* bytes);

/* Extreme Ritz values of B^-1 A (B the matrix's current preconditioner) from
 * `steps` steps of preconditioned CG on A y = r0 from y = 0: the Lanczos
 * tridiagonal T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
 * T_{j,j+1} = sqrt(beta_j)/alpha_j, whose extreme eigenvalues (bisection on
 * the Sturm count, on the device) approach the spectrum's ends from inside.
 * These are the spectral bounds the Chebyshev basis (Section IV) needs.
 * CG stops early once ||r|| <= 1e-14 ||r0||, where the Krylov space is
 * invariant to working precision (more steps would only add rounding noise).
 * r0: device FP64 vector of length n, or NULL for the library's fixed
 * pseudo-random start (splitmix64, seed 0x5EED5EED).  Errors:
 * SSCG_ERR_INVALID, SSCG_ERR_SPACE, SSCG_ERR_CUDA; SSCG_BREAKDOWN if CG
 * stops before the first step. */
int sscg_estimate_bounds(sscg_ctx* ctx, const sscg_mat* mat, int steps, const double* r0, void* workspace,
                         size_t workspace_bytes, double* lmin, double* lmax);

/* out[i] = U[-1, 1) draw i of splitmix64 started at `seed`:
 * z = mix(seed + (i+1) 0x9E3779B97F4A7C15), out = 2 (z >> 11) 2^-53 - 1.
 * A seeded device generator for start vectors and synthetic inputs. */
int sscg_uniform(sscg_ctx* ctx, int64_t n, uint64_t seed, double* out);


/* -------------------------------------------- spectral-bound network
 *
 * A learned alternative to sscg_estimate_bounds: a multilayer perceptron
 * maps ten features of the matrix to (ln lambda_min, ln lambda_max) of
 * D^-1 A (D the diagonal of A).  The paper names the Chebyshev basis
 * (Section IV) but not where its bounds come from; the features, the network
 * and its training are this library's own.  All arrays below are device
 * memory, FP64, row-major; workspaces are 256-byte aligned device memory
 * the caller owns (SSCG_ERR_SPACE when too small or misaligned).
 *
 * Network (d inputs, h hidden units per layer, o outputs):
 *   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3,
 *   theta = [W1 (h x d), b1 (h), W2 (h x h), b2 (h), W3 (o x h), b3 (o)];
 *   loss = mean over batch and outputs of (y - t)^2.
 */

/* Features, with d_i = a_ii and c_ij = |a_ij| / sqrt(d_i d_j) over the
 * nonzero off-diagonal entries:
 *   f0 = ln(n)/3, f1 = ln(nnz/n), f2 = mean ln d, f3 = std ln d,
 *   f4 = min ln d - f2, f5 = max ln d - f2, f6 = mean_i sum_{j!=i}|a_ij|/d_i,
 *   f7 = mean ln c, f8 = std ln c, f9 = min ln c  (f7-f9 are 0 without
 *   off-diagonal entries).
 * The pass reads the FP32 copies of the values and of 1/d and works in FP32
 * with FP64 sums, so each feature carries an error of about 1e-6 relative
 * (absolute near zero). */
#define SSCG_NFEAT 10
int sscg_features_workspace_bytes(size_t* bytes);
int sscg_mat_features(sscg_ctx* ctx, const sscg_mat* mat, double* feat /* SSCG_NFEAT */, void* workspace,
                      size_t workspace_bytes);

/* Parameter count h d + h + h h + h + o h + o, or -1 for a size below 1. */
int64_t sscg_mlp_nparams(int d, int h, int o);
/* Workspace for sscg_mlp_forward / _loss_grad / _train at this batch size. */
int sscg_mlp_workspace_bytes(int d, int h, int o, int batch, size_t* bytes);
/* Y (batch x o) = network(X (batch x d)).  Stream-ordered. */
int sscg_mlp_forward(sscg_ctx* ctx, int d, int h, int o, const double* theta, int batch, const double* X, double* Y,
                     void* workspace, size_t workspace_bytes);
/* grad (nparams) = d loss / d theta for targets T (batch x o), by the chain
 * rule layer by layer (tanh' = 1 - tanh^2).  When `loss` (a host pointer) is
 * not NULL the call waits and stores the loss there; otherwise it is
 * stream-ordered. */
int sscg_mlp_loss_grad(sscg_ctx* ctx, int d, int h, int o, const double* theta, int batch, const double* X,
                       const double* T, double* grad, double* loss, void* workspace, size_t workspace_bytes);
/* One Adam step (Kingma and Ba, 2015) at step t >= 1 on theta, with first
 * and second moments m, v (np each, zero before step 1):
 *   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 *   theta -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).  Stream-ordered. */
int sscg_mlp_adam_step(sscg_ctx* ctx, int64_t np, double* theta, const double* grad, double* m, double* v, double lr,
                       double beta1, double beta2, double eps, int t);
/* Full-batch training: `epochs` Adam steps (b1 0.9, b2 0.999, eps 1e-8) on
 * the mean squared error, theta updated in place.  loss_hist: device array
 * of `epochs` doubles receiving the loss before each step, or NULL.
 * Returns after the last step. */
int sscg_mlp_train(sscg_ctx* ctx, int d, int h, int o, double* theta, int batch, const double* X, const double* T,
                   int epochs, double lr, double* loss_hist, void* workspace, size_t workspace_bytes);
/* Spectral bounds from a trained network with d = SSCG_NFEAT, o = 2 and
 * 1 <= h <= 256.  model: device array [x_mean (d), x_std (d), y_mean (2),
 * y_std (2), theta]; the network sees (f - x_mean)/x_std and its outputs
 * y give lambda = exp(y y_std + y_mean).  One features pass (about the
 * traffic of one SpMV) and one inference launch; returns after the bounds
 * are on the host.  SSCG_ERR_NONFINITE if the network's interval is empty
 * or not finite (bounds untouched).  Workspace: sscg_features_workspace_bytes. */
int sscg_bounds_mlp(sscg_ctx* ctx, const sscg_mat* mat, int h, const double* model, void* workspace,
                    size_t workspace_bytes, double* lmin, double* lmax);

/* Attach a trained bounds network (the model blob of sscg_bounds_mlp, width
 * h) to a matrix, or detach it with model = NULL.  The blob is borrowed: it
 * must stay valid while attached.  A Chebyshev-basis solve given no interval
 * then takes its interval from the network instead of Lanczos steps, when
 * the matrix's preconditioner is Jacobi (the network predicts the interval
 * of D^-1 A); a network interval that is empty or not finite makes the solve
 * return SSCG_ERR_NONFINITE.  SSCG_ERR_INVALID for h outside 1..256. */
int sscg_set_bounds_model(sscg_mat* mat, int h, const double* model);


/* ------------------------------------------------------ batched solves
 *
 * Many independent SPD systems, each with 1..SSCG_BATCH_MAX_RHS right-hand
 * sides, solved together.  Every (system, right-hand side) runs Algorithm 3
 * with the monomial basis and the moment recurrence of Algorithm 6 under the
 * Jacobi preconditioner, as sscg_solve does for one system (in the z = D^-1 r,
 * Q = D^-1 A P form).  The kernels work on all systems at once: per outer
 * step, s matrix-powers levels (each gathering A's column once for all of a
 * system's right-hand sides, whose vectors are interleaved row by row), one
 * launch of per-system s x s solves, one block update.  By default each
 * phase is one launch over every system and an outer step is one CUDA graph,
 * replayed until every system is done; with SSCG_BATCH_PERSISTENT in
 * opts->flags the whole solve is one persistent cooperative launch whose
 * phases are separated by grid-wide barriers (waits bounded by %globaltimer).
 * The paper has no batched form; this is the library's serving path.
 *
 * The plan binds the matrices (not copied: they must outlive the plan), the
 * options (s <= SSCG_BATCH_MAX_S, monomial basis, f64 or df64 arithmetic
 * (df64: s <= 6),
 * tol, maxit, flags) and the caller's workspace.  Rows are processed in items
 * of T rows per system; T depends on the system's size class (n < 2^16,
 * < 2^19, < 2^21, larger).  With `tune` set, sscg_batch_create times two
 * outer steps of each class's systems (synthetic right-hand sides) for T in
 * {256, 512, 1024, 2048, 4096} and keeps the fastest; otherwise fixed
 * defaults apply.
 */
#define SSCG_BATCH_PERSISTENT 0x10u /* sscg_opts.flags: the batched solve as one cooperative launch */
#define SSCG_BATCH_MAX_RHS 8
#define SSCG_BATCH_MAX_S 8
#define SSCG_BATCH_MAX_SYSTEMS 4096
typedef struct sscg_batch sscg_batch;

/* Workspace bytes for a plan (SSCG_ERR_INVALID on bad arguments). */
int sscg_batch_workspace_bytes(int nsys, const sscg_mat* const* mats, const int* nrhs, const sscg_opts* opts,
                               size_t* bytes);
/* Create a plan.  mats[k]: the systems (Jacobi preconditioner set);
 * nrhs[k] in 1..SSCG_BATCH_MAX_RHS.  Errors: SSCG_ERR_INVALID (sizes,
 * options, preconditioner), SSCG_ERR_SPACE (workspace), SSCG_ERR_CUDA,
 * SSCG_TIMEOUT (an autotuning run stopped). */
int sscg_batch_create(sscg_ctx* ctx, int nsys, const sscg_mat* const* mats, const int* nrhs, const sscg_opts* opts,
                      int tune, void* workspace, size_t workspace_bytes, sscg_batch** plan);
int sscg_batch_destroy(sscg_batch* plan);
/* Solve all systems.  B[k], X[k]: device FP64 arrays of n_k x nrhs[k],
 * column-major (right-hand side r at offset r n_k); X holds x0 on entry and
 * the solution on exit.  infos[k] (may be NULL): per system, the worst
 * status and the largest iteration count and residuals over its right-hand
 * sides; rhs_infos (may be NULL): one entry per right-hand side, systems in
 * order; latency_ms[k] (may be NULL): device time from the kernel's start
 * until system k's result (x and true residual) was final.  hist is not
 * written.  Returns after the results are on the host: SSCG_OK, or the worst
 * positive status over all right-hand sides; SSCG_TIMEOUT if a barrier wait
 * expired (x then undefined). */
int sscg_batch_solve(sscg_batch* plan, const double* const* B, double* const* X, sscg_info* infos,
                     sscg_info* rhs_infos, double* latency_ms);
/* Plan facts: rows per item of every system (nsys entries), the grid of the
 * phase launches (the co-resident grid in the persistent mode), whether
 * solves replay a CUDA graph (an outer step; the whole solve in the
 * persistent mode), and the last solve's device time in ms (CUDA events
 * around it).  Any pointer may be NULL. */
int sscg_batch_props(const sscg_batch* plan, int* tile_rows, int* grid, int* graph, float* last_ms);
/* Fault injection for tests of the bounded waits (the paper has no
 * counterpart).  Arms the next sscg_batch_solve of a plan made with
 * SSCG_BATCH_PERSISTENT: CTA `cta` of its cooperative launch skips its
 * arrival at the first grid-wide barrier, and every barrier wait of that
 * solve gives up after `wait_ms` milliseconds (1..10000) instead of 2 s.  The
 * other CTAs' waits then expire, every CTA returns (the skipping one after a
 * bounded wait of its own), and the solve returns SSCG_TIMEOUT with X
 * undefined.  Nothing faults or hangs: the context and the plan stay usable,
 * and the knob is disarmed after that one solve.  cta = -1 disarms.
 * Errors: SSCG_ERR_INVALID (not a persistent plan, cta outside the
 * cooperative grid, wait_ms outside 1..10000). */
int sscg_batch_inject_barrier_fault(sscg_batch* plan, int cta, int wait_ms);
/* Kernels the last sscg_batch_solve ran, nodes of replayed CUDA graphs
 * included (per outer step: s levels, the solves, the update; plus the
 * initial launch); 1 in the persistent mode.  0 before the first solve.
 * SSCG_ERR_INVALID for a NULL argument. */
int sscg_batch_launches(const sscg_batch* plan, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* SSCG_H */
