"""Pins for the CPU oracle: facts the paper and the mathematics fix, checked
independently of the oracle's own code (library solvers, closed forms,
brute-force powers, invariants the paper states, the paper's printed count).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
from paper_2501_03743_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def laplace7_kron(N):
    """7-point Laplacian built as a Kronecker sum of 1-D second differences."""
    T = sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])
    I = sp.identity(N)
    return (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)).toarray()


def random_spd_csr(n, seed, density=0.3):
    """Sparse SPD matrix from the seeded generator: symmetric pattern, strictly
    diagonally dominant with a random positive diagonal."""
    u = inputs.uniform(seed, n * n).reshape(n, n)
    mask = np.abs(u) < density
    S = np.where(mask, u, 0.0)
    S = np.triu(S, 1)
    S = S + S.T
    d = np.abs(S).sum(axis=1) + 0.5 + np.abs(inputs.uniform(seed + 1, n))
    D = S + np.diag(d)
    return oracle.Matrix.from_dense(D), D


# ------------------------------------------------------------- generators

def test_splitmix64_published_vectors():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    got = [format(int(v), "016x") for v in inputs.splitmix64(g["seed"], 3)]
    assert got == g["outputs_hex"]


def test_poisson7_matches_kronecker_sum():
    rp, c, v = inputs.poisson7(5)
    D = oracle.Matrix(rp, c, v).to_dense()
    assert np.array_equal(D, laplace7_kron(5))


def test_poisson27_closed_form_spectrum():
    N = 4
    D = oracle.Matrix(*inputs.poisson27(N)).to_dense()
    ev = np.linalg.eigvalsh(D)
    lo, hi = inputs.closed_form_bounds("poisson27", N)
    assert abs(ev[0] - lo) < 1e-12 and abs(ev[-1] - hi) < 1e-12


def test_poisson7_closed_form_spectrum():
    for N in (4, 7):
        ev = np.linalg.eigvalsh(laplace7_kron(N))
        lo, hi = inputs.closed_form_bounds("poisson7", N)
        assert abs(ev[0] - lo) < 1e-12 and abs(ev[-1] - hi) < 1e-12


def test_varcoef_reduces_to_poisson_and_is_spd():
    a = inputs.varcoef7(6, 0.0, 3)
    b = inputs.poisson7(6)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    D = oracle.Matrix(*inputs.varcoef7(6, 2.0, 3)).to_dense()
    assert np.allclose(D, D.T, rtol=0, atol=0)
    assert np.linalg.eigvalsh(D)[0] > 0
    g = inputs.smoothed_field(16, 5)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12


# ------------------------------------------------------------- dense solves

def test_cholesky_matches_library_and_detects_indefinite():
    for n in (1, 3, 8, 17):
        _, D = random_spd_csr(n, 10 + n)
        B = inputs.uniform(99, 2 * n).reshape(n, 2)
        st, X = oracle.chol_solve(D, B)
        assert st == oracle.OK
        assert rel(X, np.linalg.solve(D, B)) < 1e-13
    st, _ = oracle.chol_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))
    assert st == oracle.BREAKDOWN


@pytest.mark.parametrize("solver", ["pcg", "pcgs1", "pcgs2", "pcgs3", "pcgs4", "gram3", "pfcg"])
def test_tiny_systems_match_direct_solve(solver):
    """Every solver reaches the library's direct solution on tiny SPD systems."""
    cases = [_random_diag_laplace(4, 3), random_spd_csr(60, 4)]
    for M, D in cases:
        b = inputs.uniform(7, M.n)
        xs = np.linalg.solve(D, b)
        if solver == "pcg":
            r = oracle.pcg(M, b, tol=1e-12)
        elif solver == "pfcg":
            r = oracle.pfcg(M, b, tol=1e-12)
        elif solver.startswith("pcgs"):
            r = oracle.pcgs(M, b, int(solver[-1]), tol=1e-12)
        else:
            r = oracle.pcgs_gram(M, b, int(solver[-1]), tol=1e-12)
        assert r.status == oracle.OK
        assert rel(r.x, xs) < 1e-10


def test_exhausted_krylov_space_is_reported_as_breakdown():
    """The 4^3 Laplacian has 16 distinct eigenvalues, so CG ends after 16
    steps.  With s = 3 the sixth block has one dimension left, W is singular
    and the oracle stops with BREAKDOWN instead of returning garbage; with
    s = 4 the space ends on a block boundary and the run converges."""
    M = oracle.Matrix(*inputs.poisson7(4))
    b = inputs.uniform(7, M.n)
    assert oracle.pcg(M, b, tol=1e-13).iters == 16
    r3 = oracle.pcgs(M, b, 3, tol=1e-12)
    assert r3.status == oracle.BREAKDOWN and r3.iters == 5
    r4 = oracle.pcgs(M, b, 4, tol=1e-12)
    assert r4.status == oracle.OK and r4.iters == 4


# ------------------------------------------------- exact-arithmetic identities

def test_s1_is_pcg():
    """Algorithm 3 with s = 1 is Algorithm 1: same iterates, same count."""
    A = inputs.system("poisson7", 8, seed=2)
    M = oracle.as_matrix(A)
    a = oracle.pcg(M, A["b"], tol=1e-10)
    b = oracle.pcgs(M, A["b"], 1, tol=1e-10)
    assert a.iters == b.iters
    assert rel(b.x, a.x) < 1e-13
    assert np.allclose(a.hist, b.hist, rtol=1e-10, atol=0)


def _random_diag_laplace(N, seed):
    D = laplace7_kron(N) + np.diag(1.0 + np.abs(inputs.uniform(seed, N ** 3)))
    return oracle.Matrix.from_dense(D), D


@pytest.mark.parametrize("s", [2, 3, 4])
@pytest.mark.parametrize("variant", ["literal", "gram-monomial", "gram-chebyshev", "gram-newton"])
def test_block_equivalence_with_pcg(s, variant):
    """The s-step iterate x_i lies in x_0 + K_{is} and minimises the A-norm
    error there (Section II-A), so it equals PCG's x_{is}."""
    for M, _ in [_random_diag_laplace(6, 11), (oracle.Matrix(*inputs.poisson7(8)), None)]:
        b = inputs.uniform(5, M.n)
        steps = 4
        if variant == "literal":
            q = oracle.pcgs(M, b, s, tol=0.0, maxit=steps, trace=steps)
        else:
            d = oracle.diag(M)
            ev = np.linalg.eigvalsh(np.diag(d ** -0.5) @ M.to_dense() @ np.diag(d ** -0.5))
            basis = variant.split("-")[1]
            q = oracle.pcgs_gram(M, b, s, basis=basis, bounds=(ev[0] * 0.9, ev[-1] * 1.05), tol=0.0,
                                 maxit=steps, trace=steps)
        assert q.iters == steps
        for i in range(steps):
            p = oracle.pcg(M, b, tol=0.0, maxit=(i + 1) * s)
            assert p.iters == (i + 1) * s
            assert rel(q.extra["x"][i], p.x) < 1e-10, (i, rel(q.extra["x"][i], p.x))


@pytest.mark.parametrize("s", [2, 3, 4])
def test_outer_count_is_ceil_of_pcg_count(s):
    A = inputs.system("poisson7", 10, seed=1)
    M = oracle.as_matrix(A)
    k = oracle.pcg(M, A["b"], tol=1e-9).iters
    q = oracle.pcgs(M, A["b"], s, tol=1e-9)
    assert q.status == oracle.OK
    assert q.iters == -(-k // s)


def test_exact_termination_with_s_distinct_eigenvalues():
    """With B = I and s distinct eigenvalues, K_s holds the solution: one outer step."""
    n = 40
    Q, _ = np.linalg.qr(inputs.uniform(3, n * n).reshape(n, n))
    lam = np.array([1.0, 2.0, 5.0])[np.arange(n) % 3]
    D = (Q * lam) @ Q.T
    D = 0.5 * (D + D.T)
    M = oracle.Matrix.from_dense(D)
    b = inputs.uniform(4, n)
    r = oracle.pcgs(M, b, 3, prec="none", tol=1e-12)
    assert r.status == oracle.OK and r.iters == 1
    assert rel(r.x, np.linalg.solve(D, b)) < 1e-12


def test_pcg_terminates_within_n_steps():
    for n in (5, 12, 20):
        M, D = random_spd_csr(n, 30 + n, density=0.6)
        b = inputs.uniform(8, n)
        r = oracle.pcg(M, b, tol=1e-10)
        assert r.status == oracle.OK and r.iters <= n + 3


def test_pfcg_matches_pcg_for_fixed_preconditioner():
    """Notay's flexible CG (Algorithm 2) with a fixed SPD B is PCG in exact arithmetic."""
    A = inputs.system("varcoef7", 10, seed=3, sigma=1.0)
    M = oracle.as_matrix(A)
    a = oracle.pcg(M, A["b"], tol=1e-10)
    f = oracle.pfcg(M, A["b"], tol=1e-10)
    assert abs(a.iters - f.iters) <= 1
    assert rel(f.x, a.x) < 1e-8


def test_gram_variant_matches_literal_variant():
    A = inputs.system("poisson7", 12, seed=4)
    M = oracle.as_matrix(A)
    for s in (2, 4):
        a = oracle.pcgs(M, A["b"], s, tol=1e-10)
        g = oracle.pcgs_gram(M, A["b"], s, tol=1e-10)
        assert a.iters == g.iters
        assert rel(g.x, a.x) < 1e-9


# ------------------------------------------------ invariants of Section II-A

@pytest.mark.parametrize("s", [2, 3, 4])
def test_sstep_invariants(s):
    M, D = _random_diag_laplace(5, 21)
    b = inputs.uniform(6, M.n)
    steps = 5
    q = oracle.pcgs(M, b, s, tol=0.0, maxit=steps, trace=steps)
    t = q.extra
    d = np.diag(D)
    Binv = np.diag(1.0 / d)
    r_prev = b.copy()
    for i in range(steps):
        U, AU, P, AP, W = t["U"][i], t["AU"][i], t["P"][i], t["AP"][i], t["W"][i]
        # pMPK: U_j = (B^-1 A)^(j-1) B^-1 r, AU = A U (Algorithm 4)
        u = Binv @ r_prev
        for j in range(s):
            assert rel(U[:, j], u) < 1e-9
            assert rel(AU[:, j], D @ u) < 1e-9
            u = Binv @ (D @ u)
        # cvm: vm(k) = mu_{k-1} = r^T (B^-1 A)^(k-1) B^-1 r (Eq. mommat, Algorithm 5)
        z = Binv @ r_prev
        mu = [r_prev @ np.linalg.matrix_power(Binv @ D, k) @ z for k in range(2 * s)]
        assert np.allclose(t["vm"][i], mu, rtol=1e-9, atol=1e-12 * abs(mu[0]))
        # W = P^T A P, symmetric positive definite (Section II-A)
        assert rel(W, P.T @ D @ P) < 1e-8
        assert np.linalg.eigvalsh(0.5 * (W + W.T))[0] > 0
        r_new = t["r"][i]
        assert np.linalg.norm(r_new - (b - D @ t["x"][i])) / np.linalg.norm(b) < 1e-13
        # r_{i+1} is orthogonal to the new directions (Eq. normaleq)
        assert np.linalg.norm(P.T @ r_new) / (np.linalg.norm(P) * np.linalg.norm(r_new)) < 1e-8
        if i > 0:
            Pold, APold = t["P"][i - 1], t["AP"][i - 1]
            # block A-conjugacy W_{i-1} beta + c = 0 holds (Section II-A)
            assert np.linalg.norm(Pold.T @ D @ P) / np.linalg.norm(W) < 1e-8
            # c = (A P_old)^T U is Hankel with zeros for l + j <= s, and b1 = -c (Algorithm 6)
            Cm = APold.T @ U
            scale = np.abs(Cm).max()
            for l in range(s):
                for j in range(s):
                    if l + j + 2 <= s:
                        assert abs(Cm[l, j]) < 1e-8 * scale
                    if l + 1 < s and j > 0:
                        assert abs(Cm[l + 1, j - 1] - Cm[l, j]) < 1e-8 * scale
            assert np.abs(t["b1"][i] + Cm).max() < 1e-8 * scale
            # W_i = M_i - c_i beta_{i-1} with the Hankel moment matrix M_i
            H = np.array([[t["vm"][i][a + c + 1] for c in range(s)] for a in range(s)])
            assert rel(W, H - t["b1"][i] @ t["beta"][i]) < 1e-12
        r_prev = r_new


def test_literal_b1_bound_breaks_conjugacy():
    """Reading check for Algorithm 6: b1 filled only for j < i leaves P_old^T A P
    far from zero, so the full fill is the consistent reading."""
    M, D = _random_diag_laplace(5, 21)
    b = inputs.uniform(6, M.n)
    s = 3
    q = oracle.pcgs(M, b, s, tol=0.0, maxit=3, trace=3)
    t = q.extra
    b1 = t["b1"][1]
    lower = np.tril(b1, -1)
    Wold = t["W"][0]
    beta_lit = np.linalg.solve(Wold, lower)
    P_lit = t["U"][1] + t["P"][0] @ beta_lit
    P_ok = t["P"][1]
    Pold = t["P"][0]
    assert np.linalg.norm(Pold.T @ D @ P_ok) / np.linalg.norm(P_ok.T @ D @ P_ok) < 1e-8
    assert np.linalg.norm(Pold.T @ D @ P_lit) / np.linalg.norm(P_lit.T @ D @ P_lit) > 1e-3


# ------------------------------------------------ spectra, bounds, polynomials

def test_tridiagonal_extremes_match_library():
    d = 2.0 + inputs.uniform(40, 30)
    e = inputs.uniform(41, 29)
    lo, hi = oracle.tridiag_extremes(d, e)
    ev = sla.eigvalsh_tridiagonal(d, e)
    assert abs(lo - ev[0]) < 1e-12 and abs(hi - ev[-1]) < 1e-12


def test_lanczos_bounds_reach_closed_form():
    """Ritz extremes of D^-1 A for the 7-point stencil converge to
    (6 -/+ 6 cos(pi/(N+1)))/6."""
    N = 10
    A = inputs.system("poisson7", N, seed=0)
    lo, hi = oracle.lanczos_bounds(oracle.as_matrix(A), inputs.uniform(9, N ** 3), 120)
    clo, chi = inputs.closed_form_bounds("poisson7", N)
    assert abs(hi - chi / 6) < 1e-8 and abs(lo - clo / 6) < 1e-6
    # few steps: Ritz values lie inside the spectrum
    lo5, hi5 = oracle.lanczos_bounds(oracle.as_matrix(A), inputs.uniform(9, N ** 3), 5)
    assert clo / 6 - 1e-12 <= lo5 and hi5 <= chi / 6 + 1e-12


def test_lanczos_full_run_gives_exact_extremes():
    M, D = random_spd_csr(25, 77, density=0.5)
    d = np.diag(D)
    ev = np.linalg.eigvalsh(np.diag(d ** -0.5) @ D @ np.diag(d ** -0.5))
    lo, hi = oracle.lanczos_bounds(M, inputs.uniform(2, 25), 25)
    assert abs(lo - ev[0]) < 1e-8 and abs(hi - ev[-1]) < 1e-8


def test_lanczos_more_steps_than_needed_stays_in_spectrum():
    """Asking for far more steps than CG needs (27-point stencil, kappa ~ 23,
    400 steps on 1,728 unknowns) still gives Ritz values at the exact ends of
    the spectrum of D^-1 A: no spurious values from steps past convergence."""
    N = 12
    A = inputs.system("poisson27", N, seed=0)
    lo, hi = oracle.lanczos_bounds(oracle.as_matrix(A), inputs.uniform(3, N ** 3), 400)
    clo, chi = inputs.closed_form_bounds("poisson27", N)
    assert abs(lo - clo / 26) < 1e-7 * chi and abs(hi - chi / 26) < 1e-7 * chi


def _cheb_T(m, x):
    x = np.asarray(x, dtype=float)
    inside = np.cos(m * np.arccos(np.clip(x, -1, 1)))
    outside = np.sign(x) ** m * np.cosh(m * np.arccosh(np.maximum(np.abs(x), 1.0)))
    return np.where(np.abs(x) <= 1, inside, outside)


@pytest.mark.parametrize("degree", [1, 2, 3, 5])
def test_chebyshev_preconditioner_residual_polynomial(degree):
    """For an eigenvector v of D^-1 A with eigenvalue lam, B^-1 A v =
    (1 - T_m((theta - lam)/delta) / T_m(theta/delta)) v."""
    N = 6
    M = oracle.Matrix(*inputs.poisson7(N))
    i = np.arange(N)
    k = (1, 2, 4)
    v = np.einsum("a,b,c->abc", *[np.sin((kk * (i + 1) * np.pi) / (N + 1)) for kk in k[::-1]]).reshape(-1)
    lam = sum(2 - 2 * np.cos(kk * np.pi / (N + 1)) for kk in k) / 6
    lmin, lmax = 0.05, 1.97
    z = oracle.prec_apply(M, dict(kind="cheb", degree=degree, lmin=lmin, lmax=lmax), oracle.spmv(M, v))
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    factor = 1 - _cheb_T(degree, (theta - lam) / delta) / _cheb_T(degree, theta / delta)
    assert rel(z, factor * v) < 1e-12


def _laplace_modes(N, ks):
    """Sine eigenvectors of the 7-point stencil and their eigenvalues of D^-1 A."""
    i = np.arange(N)
    vs, lams = [], []
    for k in ks:
        v = np.einsum("a,b,c->abc", *[np.sin((kk * (i + 1) * np.pi) / (N + 1)) for kk in k[::-1]]).reshape(-1)
        vs.append(v / np.linalg.norm(v))
        lams.append(sum(2 - 2 * np.cos(kk * np.pi / (N + 1)) for kk in k) / 6)
    return vs, lams


@pytest.mark.parametrize("basis", ["monomial", "chebyshev", "newton"])
def test_basis_vectors_closed_form(basis):
    """With b = A sum_k v_k over eigenvectors of D^-1 A (Jacobi, x0 = 0),
    z = D^-1 b = sum_k lam_k v_k and the basis vectors are
    u_j = sum_k lam_k q_{j-1}(lam_k) v_k with q_m(l) = l^m (monomial),
    T_m((l - c)/delta) (Chebyshev, T_m(x) = cos(m arccos x)) or
    prod_{i<m} (l - theta_i) / sigma (Newton, the oracle's shifts)."""
    N, s = 7, 4
    vs, lams = _laplace_modes(N, [(1, 1, 1), (1, 2, 1), (2, 2, 3), (3, 1, 4), (5, 4, 2), (6, 6, 6)])
    M = oracle.Matrix(*inputs.poisson7(N))
    b = oracle.spmv(M, sum(vs))
    lo, hi = 0.05, 1.96
    c, delta = (lo + hi) / 2, (hi - lo) / 2
    q = oracle.pcgs_gram(M, b, s, basis=basis, bounds=(lo, hi), tol=0.0, maxit=1, trace=1)
    U = q.extra["U"][0]
    for j in range(s):
        if basis == "monomial":
            want = sum(l * l ** j * v for l, v in zip(lams, vs))
        elif basis == "chebyshev":
            want = sum(l * _cheb_T(j, (l - c) / delta) * v for l, v in zip(lams, vs))
        else:
            th, sig = oracle.newton_shifts(s, lo, hi)
            want = sum(l * np.prod([(l - t) / sig for t in th[:j]]) * v for l, v in zip(lams, vs))
        assert rel(U[:, j], want) < 1e-12


@pytest.mark.parametrize("s", [2, 3, 5, 8, 12])
def test_newton_shifts_are_leja_ordered_chebyshev_points(s):
    """The shifts are the zeros of T_{s-1} on [lo, hi] (numpy's Chebyshev
    roots), in Leja order: the first of largest modulus, each next maximising
    the product of its distances to the earlier ones (checked by brute force
    over the remaining points); sigma = (hi - lo)/4 is the interval's
    capacity: the monic polynomial with these zeros has sup norm 2 sigma^m
    on [lo, hi]."""
    lo, hi = 0.07, 2.3
    th, sig = oracle.newton_shifts(s, lo, hi)
    m = s - 1
    assert len(th) == m
    if m == 0:
        return
    c, d = (lo + hi) / 2, (hi - lo) / 2
    roots = np.sort(np.real(c + d * np.polynomial.chebyshev.Chebyshev.basis(m).roots()))
    assert np.allclose(np.sort(th), roots, rtol=0, atol=1e-13)
    assert abs(th[0]) == max(abs(th))
    for q in range(1, m):
        rest = th[q:]  # the points not chosen before step q
        score = [np.prod(np.abs(t - th[:q])) for t in rest]
        assert np.prod(np.abs(th[q] - th[:q])) >= max(score) * (1 - 1e-12)
    assert sig == pytest.approx((hi - lo) / 4, rel=1e-15)
    xs = np.linspace(lo, hi, 200001)
    sup = np.max(np.abs(np.prod(xs[:, None] - th[None, :], axis=1)))
    assert sup == pytest.approx(2 * sig ** m, rel=1e-6)


def test_newton_basis_converges_where_monomial_breaks_down():
    """Section IV: Newton (like Chebyshev) bases keep large blocks usable."""
    A = inputs.system("varcoef7", 10, seed=2, sigma=1.0)
    M = oracle.as_matrix(A)
    d = oracle.diag(M)
    ev = np.linalg.eigvalsh(np.diag(d ** -0.5) @ M.to_dense() @ np.diag(d ** -0.5))
    mono = oracle.pcgs(M, A["b"], 12, tol=1e-10, maxit=200)
    newt = oracle.pcgs_gram(M, A["b"], 12, basis="newton", bounds=(ev[0] * 0.95, ev[-1] * 1.05), tol=1e-10,
                            maxit=200)
    assert mono.status != oracle.OK
    assert newt.status == oracle.OK
    ref = oracle.pcg(M, A["b"], tol=1e-12)
    assert rel(newt.x, ref.x) < 1e-8


def test_jacobi_pcg_equals_cg_for_constant_stencil():
    """D = 6 I, so Jacobi-PCG produces CG's iterates: equal counts and x."""
    A = inputs.system("poisson7", 12, seed=5)
    M = oracle.as_matrix(A)
    a = oracle.pcg(M, A["b"], prec="jacobi", tol=1e-10)
    b = oracle.pcg(M, A["b"], prec="none", tol=1e-10)
    assert a.iters == b.iters and rel(a.x, b.x) < 1e-12


def test_convergence_bound():
    """CG needs at most (1/2) sqrt(kappa) ln(2/tol) iterations."""
    for N in (12, 24):
        A = inputs.system("poisson7", N, seed=0)
        lo, hi = inputs.closed_form_bounds("poisson7", N)
        tol = 1e-8
        bound = 0.5 * np.sqrt(hi / lo) * np.log(2 / tol)
        r = oracle.pcg(oracle.as_matrix(A), A["b"], tol=tol)
        assert r.status == oracle.OK and r.iters <= bound


@pytest.mark.parametrize("s", [1, 2, 4])
def test_residual_gap_at_convergence(s):
    A = inputs.system("poisson7", 16, seed=6)
    M = oracle.as_matrix(A)
    q = oracle.pcgs(M, A["b"], s, tol=1e-8)
    true = np.linalg.norm(A["b"] - oracle.spmv(M, q.x)) / np.linalg.norm(A["b"])
    assert q.status == oracle.OK and abs(true - q.relres) < 1e-10


def test_monomial_instability_at_large_s():
    """Section II-A warns the monomial basis loses independence as s grows:
    at s = 10 on 16^3 the run breaks down or needs extra outer steps."""
    A = inputs.system("poisson7", 16, seed=0)
    M = oracle.as_matrix(A)
    k = oracle.pcg(M, A["b"], tol=1e-8).iters
    q = oracle.pcgs(M, A["b"], 10, tol=1e-8, maxit=200)
    assert q.status != oracle.OK or q.iters > -(-k // 10)


# ------------------------------------------------------------------ MLP

def test_mlp_gradient_matches_finite_differences():
    d, h, o = 6, 9, 2
    npar = oracle.mlp_nparams(d, h, o)
    theta = 0.4 * inputs.uniform(1, npar)
    X = inputs.uniform(2, 5 * d).reshape(5, d)
    T = inputs.uniform(3, 5 * o).reshape(5, o)
    loss, g = oracle.mlp_loss_grad(d, h, o, theta, X, T)
    fd = np.zeros(npar)
    eps = 1e-6
    for i in range(npar):
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd[i] = (oracle.mlp_loss_grad(d, h, o, tp, X, T)[0] - oracle.mlp_loss_grad(d, h, o, tm, X, T)[0]) / (2 * eps)
    assert rel(g, fd) < 1e-7
    Y = oracle.mlp_forward(d, h, o, theta, X)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-14


def test_mlp_forward_special_case():
    """With W1 = W2 = 0 the output is W3 tanh(b2) + b3 for every input."""
    d, h, o = 4, 5, 2
    theta = np.zeros(oracle.mlp_nparams(d, h, o))
    b2 = np.linspace(-1, 1, h)
    W3 = np.arange(o * h, dtype=float).reshape(o, h)
    b3 = np.array([0.5, -0.25])
    off = h * d + h + h * h
    theta[off:off + h] = b2
    theta[off + h:off + h + o * h] = W3.reshape(-1)
    theta[off + h + o * h:] = b3
    Y = oracle.mlp_forward(d, h, o, theta, inputs.uniform(0, 3 * d).reshape(3, d))
    assert np.allclose(Y, (W3 @ np.tanh(b2) + b3)[None, :], rtol=1e-15, atol=1e-15)


# ------------------------------------------------- features and optimiser

def test_features_closed_form_poisson7():
    """Constant 7-point stencil on N^3: every diagonal is 6 and every coupling
    |a_ij|/sqrt(d_i d_j) is 1/6, so the spreads vanish; nnz = 7n - 6N^2."""
    N = 5
    A = inputs.system("poisson7", N, seed=0)
    n = N ** 3
    nnz = 7 * n - 6 * N * N
    assert int(A["rowptr"][-1]) == nnz
    f = oracle.features(A)
    want = [np.log(N), np.log(nnz / n), np.log(6.0), 0.0, 0.0, 0.0, (nnz - n) / (6.0 * n),
            np.log(1 / 6), 0.0, np.log(1 / 6)]
    assert np.allclose(f, want, rtol=1e-13, atol=1e-13)


def test_features_closed_form_poisson27():
    N = 4
    A = inputs.system("poisson27", N, seed=0)
    n = N ** 3
    nnz = int(A["rowptr"][-1])
    assert nnz == (3 * N - 2) ** 3  # a 1-D factor of N + 2(N-1) entries per direction
    f = oracle.features(A)
    assert np.allclose(f[[2, 7, 9]], [np.log(26.0), np.log(1 / 26), np.log(1 / 26)], rtol=1e-13)
    assert np.allclose(f[[3, 4, 5, 8]], 0.0, atol=1e-13)
    assert abs(f[6] - (nnz - n) / (26.0 * n)) < 1e-14


def test_features_two_valued_diagonal():
    """Diagonal matrix with entries e^a and e^b, two of each: mean (a+b)/2,
    standard deviation |a-b|/2; no off-diagonal entries."""
    a, b = -0.7, 1.9
    D = np.diag(np.exp([a, b, b, a]))
    f = oracle.features(oracle.Matrix.from_dense(D))
    want = [np.log(4) / 3, 0.0, (a + b) / 2, (b - a) / 2, -(b - a) / 2, (b - a) / 2, 0.0, 0.0, 0.0, 0.0]
    assert np.allclose(f, want, rtol=1e-13, atol=1e-13)


def test_features_scaling_invariances():
    """Scaling A by c shifts the mean log-diagonal by ln c and leaves the rest;
    a symmetric diagonal scaling S A S leaves the couplings (f7-f9) alone."""
    _, D = random_spd_csr(30, seed=11)
    f = oracle.features(oracle.Matrix.from_dense(D))
    g = oracle.features(oracle.Matrix.from_dense(3.5 * D))
    assert abs(g[2] - f[2] - np.log(3.5)) < 1e-13
    assert np.allclose(np.delete(g, 2), np.delete(f, 2), rtol=1e-12, atol=1e-13)
    s = np.exp(inputs.uniform(12, 30))
    h = oracle.features(oracle.Matrix.from_dense(D * s[:, None] * s[None, :]))
    assert np.allclose(h[7:], f[7:], rtol=1e-12, atol=1e-13)
    assert abs(h[2] - f[2] - 2 * np.mean(np.log(s))) < 1e-12
    # the coupling of a 2x2 block [[p, q], [q, r]] is |q|/sqrt(pr)
    t = oracle.features(oracle.Matrix.from_dense(np.array([[4.0, -1.0], [-1.0, 9.0]])))
    assert np.allclose(t[7:], [np.log(1 / 6), 0.0, np.log(1 / 6)], rtol=1e-14)
    assert abs(t[6] - (1 / 4 + 1 / 9) / 2) < 1e-15


def test_adam_constant_gradient_closed_form():
    """With a constant gradient the bias-corrected moments equal g and g^2, so
    every step moves theta by lr g / (|g| + eps)."""
    g = inputs.uniform(5, 7)
    theta = inputs.uniform(6, 7)
    t0 = theta.copy()
    m, v = np.zeros(7), np.zeros(7)
    for t in range(1, 6):
        oracle.adam_step(theta, g, m, v, t, lr=0.01)
    assert np.allclose(theta, t0 - 5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=1e-15)


def test_adam_alternating_gradient_closed_form():
    """Gradients g then -g: after two steps m/(1-b1^2) = -(1-b1)/(1+b1) g and
    v/(1-b2^2) = g^2, so the second step moves by +lr (1-b1)/(1+b1) g/(|g|+eps)."""
    b1, b2, lr, eps = 0.8, 0.95, 0.1, 1e-8
    g = inputs.uniform(7, 5)
    theta = np.zeros(5)
    m, v = np.zeros(5), np.zeros(5)
    oracle.adam_step(theta, g, m, v, 1, lr, b1, b2, eps)
    after1 = theta.copy()
    assert np.allclose(after1, -lr * g / (np.abs(g) + eps), rtol=1e-14)
    oracle.adam_step(theta, -g, m, v, 2, lr, b1, b2, eps)
    assert np.allclose(theta - after1, lr * (1 - b1) / (1 + b1) * g / (np.abs(g) + eps), rtol=1e-12)


# ------------------------------------------------------- the paper's count

@pytest.mark.slow
def test_paper_iteration_count_250():
    """Section VI: 250^3 Poisson, b = 1, rtol 1e-6, no preconditioner:
    PCGs with s = 1 (equal to PCG, pinned above) takes 514 iterations."""
    g = json.load(open(os.path.join(GOLDEN, "paper_iterations.json")))
    M = oracle.Matrix(*inputs.poisson7(g["N"]))
    r = oracle.pcg(M, np.ones(M.n), prec="none", tol=g["rtol"], maxit=g["itmax"])
    assert r.status == oracle.OK
    assert r.iters == g["iterations"]
