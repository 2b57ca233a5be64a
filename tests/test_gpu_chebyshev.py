"""Parity of the direct-Gram s-step path (Chebyshev basis, Chebyshev
polynomial preconditioner), the Lanczos bound estimate and the device
generator with the FP64 oracle and closed forms, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2501_03743_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_03743_gb300 import sscg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_2501_03743_gb300 import build

    build.build()
    return sscg.Context()


_CACHE = {}


def system(kind, N, seed=0, sigma=0.0):
    key = (kind, N, seed, sigma)
    if key not in _CACHE:
        _CACHE[key] = inputs.system(kind, N, seed=seed, sigma=sigma)
    return _CACHE[key]


def gpu_matrix(ctx, S):
    return sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])


def gpu_solve(A, b, method="sstep", **kw):
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.zeros_like(bt)
    res = sscg.Solver(A, method=method, **kw).solve(bt, xt)
    return xt.cpu().numpy(), res


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_device_generator_matches_published_definition(ctx):
    for seed in (0, 12345, 2 ** 63 + 7):
        got = ctx.uniform(1000, seed).cpu().numpy()
        assert np.array_equal(got, inputs.uniform(seed, 1000))


@pytest.mark.parametrize("N", [10, 17])
def test_lanczos_bounds_match_oracle_and_closed_form(ctx, N):
    S = system("poisson7", N)
    A = gpu_matrix(ctx, S)
    r0 = inputs.uniform(9, S["n"])
    for k in (5, 20, 60):
        lo, hi = A.estimate_bounds(k, torch.from_numpy(r0).cuda())
        olo, ohi = oracle.lanczos_bounds(oracle.as_matrix(S), r0, k)
        assert abs(lo - olo) < 1e-6 * ohi and abs(hi - ohi) < 1e-6 * ohi
        clo, chi = inputs.closed_form_bounds("poisson7", N)
        assert clo / 6 - 1e-9 <= lo <= hi <= chi / 6 + 1e-9  # Ritz values lie inside the spectrum
    assert abs(hi - chi / 6) < 1e-6


def test_lanczos_default_start(ctx):
    S = system("varcoef7", 12, 2, 2.0)
    A = gpu_matrix(ctx, S)
    lo, hi = A.estimate_bounds(30)
    olo, ohi = oracle.lanczos_bounds(oracle.as_matrix(S), inputs.uniform(0x5EED5EED, S["n"]), 30)
    assert abs(lo - olo) < 1e-6 * ohi and abs(hi - ohi) < 1e-6 * ohi


def _jacobi_bounds(S):
    M = oracle.as_matrix(S)
    lo, hi = oracle.lanczos_bounds(M, inputs.uniform(1, S["n"]), 60)
    return 0.95 * lo, 1.05 * hi


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("s", [2, 4, 8, 12])
def test_chebyshev_basis_parity(ctx, arith, s):
    S = system("varcoef7", 14, 3, 2.0)
    A = gpu_matrix(ctx, S)
    bnd = _jacobi_bounds(S)
    x, res = gpu_solve(A, S["b"], s=s, basis="chebyshev", basis_bounds=bnd, tol=1e-8, maxit=500, arith=arith)
    ref = oracle.pcgs_gram(oracle.as_matrix(S), S["b"], s, basis="chebyshev", bounds=bnd, tol=1e-8, maxit=500)
    assert ref.status == oracle.OK
    assert res.status == sscg.OK and res.rel_res_recursive < 1e-8
    assert abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pcgs_gram(oracle.as_matrix(S), S["b"], s, basis="chebyshev", bounds=bnd, tol=0.0,
                            maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7
    assert res.rel_res_true < 10 * 1e-8


def test_chebyshev_basis_automatic_bounds(ctx):
    """With no interval given the solve estimates one by 20 Lanczos steps."""
    S = system("poisson7", 20, 1)
    A = gpu_matrix(ctx, S)
    x, res = gpu_solve(A, S["b"], s=8, basis="chebyshev", tol=1e-8, maxit=300)
    assert res.status == sscg.OK and res.rel_res_true < 1e-7
    k = oracle.pcg(oracle.as_matrix(S), S["b"], tol=1e-8).iters
    assert res.outer_iters <= -(-k // 8) + 1
    assert rel(x, S["x_true"]) < 1e-5


@pytest.mark.parametrize("s", [2, 4])
def test_direct_gram_monomial_matches_both_oracles(ctx, s):
    S = system("poisson7", 15, 4)
    A = gpu_matrix(ctx, S)
    x, res = gpu_solve(A, S["b"], s=s, tol=1e-8, maxit=500, direct_gram=True)
    ref = oracle.pcgs_gram(oracle.as_matrix(S), S["b"], s, tol=1e-8, maxit=500)
    lit = oracle.pcgs(oracle.as_matrix(S), S["b"], s, tol=1e-8, maxit=500)
    assert res.status == sscg.OK and abs(res.outer_iters - ref.iters) <= 1 and abs(res.outer_iters - lit.iters) <= 1
    same = oracle.pcgs_gram(oracle.as_matrix(S), S["b"], s, tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7


@pytest.mark.parametrize("degree", [1, 2, 4])
def test_chebyshev_preconditioner_pcg_parity(ctx, degree):
    S = system("varcoef7", 13, 6, 1.0)
    A = gpu_matrix(ctx, S)
    lo, hi = _jacobi_bounds(S)
    A.set_preconditioner("cheb", degree, lo, hi)
    prec = dict(kind="cheb", degree=degree, lmin=lo, lmax=hi)
    for arith in ("f64", "df64"):
        x, res = gpu_solve(A, S["b"], method="pcg", tol=1e-8, maxit=2000, arith=arith)
        ref = oracle.pcg(oracle.as_matrix(S), S["b"], prec=prec, tol=1e-8, maxit=2000)
        assert res.status == sscg.OK and abs(res.outer_iters - ref.iters) <= 1
        same = oracle.pcg(oracle.as_matrix(S), S["b"], prec=prec, tol=0.0, maxit=res.outer_iters)
        assert rel(x, same.x) < 1e-7


@pytest.mark.parametrize("basis", ["monomial", "chebyshev"])
def test_chebyshev_preconditioner_sstep_parity(ctx, basis):
    S = system("varcoef7", 13, 6, 1.0)
    A = gpu_matrix(ctx, S)
    lo, hi = _jacobi_bounds(S)
    degree = 3
    A.set_preconditioner("cheb", degree, lo, hi)
    prec = dict(kind="cheb", degree=degree, lmin=lo, lmax=hi)
    # B^-1 A has its spectrum in [1 - eps, 1 + eps], eps = 1/T_3(theta/delta)
    th, de = (hi + lo) / 2, (hi - lo) / 2
    eps = 1.0 / np.cosh(degree * np.arccosh(th / de))
    bnd = (1 - 1.05 * eps, 1 + 1.05 * eps)
    s = 4
    x, res = gpu_solve(A, S["b"], s=s, basis=basis, basis_bounds=bnd, tol=1e-8, maxit=500)
    ref = oracle.pcgs_gram(oracle.as_matrix(S), S["b"], s, basis=basis, bounds=bnd, prec=prec, tol=1e-8, maxit=500)
    assert res.status == sscg.OK and abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pcgs_gram(oracle.as_matrix(S), S["b"], s, basis=basis, bounds=bnd, prec=prec, tol=0.0,
                            maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7


def test_chebyshev_basis_stays_stable_where_monomial_fails(ctx):
    """Section IV: the Chebyshev basis keeps large s usable."""
    S = system("poisson7", 24, 2)
    A = gpu_matrix(ctx, S)
    xm, rm = gpu_solve(A, S["b"], s=12, tol=1e-8, maxit=300)
    xc, rc = gpu_solve(A, S["b"], s=12, basis="chebyshev", tol=1e-8, maxit=300)
    assert rc.status == sscg.OK
    assert rm.status != sscg.OK or rm.outer_iters > rc.outer_iters
