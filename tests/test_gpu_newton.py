"""The Newton basis (Leja-ordered Chebyshev points of the spectral interval
as shifts) and the adaptive block size on the GPU, through the C ABI: parity
with the FP64 oracle's direct-Gram s-step method with the same basis, the
diagonal form against CSR, the mixed-precision mode, automatic intervals,
and restarts with s halved after a breakdown."""
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


def solve(A, b, **kw):
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.zeros_like(bt)
    res = sscg.Solver(A, **kw).solve(bt, xt)
    return xt.cpu().numpy(), res


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def jacobi_interval(S):
    lo, hi = oracle.lanczos_bounds(oracle.as_matrix(S), inputs.uniform(1, S["n"]), 60)
    return 0.95 * lo, 1.05 * hi


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("s", [2, 4, 8, 12])
def test_newton_basis_parity(ctx, arith, s):
    S = system("varcoef7", 14, 3, 2.0)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    bnd = jacobi_interval(S)
    M = oracle.as_matrix(S)
    x, res = solve(A, S["b"], s=s, basis="newton", basis_bounds=bnd, tol=1e-8, maxit=500, arith=arith)
    ref = oracle.pcgs_gram(M, S["b"], s, basis="newton", bounds=bnd, tol=1e-8, maxit=500)
    assert ref.status == oracle.OK
    assert res.status == sscg.OK and res.rel_res_recursive < 1e-8 and res.rel_res_true < 1e-7
    assert abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pcgs_gram(M, S["b"], s, basis="newton", bounds=bnd, tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7


@pytest.mark.parametrize("kind,N", [("poisson7", 19), ("aniso7", 15), ("poisson27", 11)])
def test_newton_basis_diagonal_form_matches_csr(ctx, kind, N):
    S = system(kind, N, 5)
    Ad = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    Ac = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"], csr_only=True)
    bnd = jacobi_interval(S)
    for arith in ("df64", "f64"):
        xd, rd = solve(Ad, S["b"], s=6, basis="newton", basis_bounds=bnd, tol=1e-9, maxit=1000, arith=arith)
        xc, rc = solve(Ac, S["b"], s=6, basis="newton", basis_bounds=bnd, tol=1e-9, maxit=1000, arith=arith)
        assert rd.status == rc.status == sscg.OK and rd.outer_iters == rc.outer_iters
        assert rel(xd, xc) < 1e-10


def test_newton_basis_in_mixed_precision(ctx):
    S = system("poisson27", 20, 1)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    bnd = jacobi_interval(S)
    x, res = solve(A, S["b"], s=8, basis="newton", basis_bounds=bnd, tol=1e-10, maxit=1000, arith="mixed",
                   replace_every=1)
    assert res.status == sscg.OK and res.rel_res_true < 2e-10
    ref = oracle.pcg(oracle.as_matrix(S), S["b"], tol=1e-10, maxit=5000)
    assert rel(x, ref.x) < 1e-7


def test_newton_basis_automatic_interval_and_large_s(ctx):
    """With no interval the solve estimates one (20 Lanczos steps); at s = 12
    the Newton basis converges where the monomial basis breaks down."""
    S = system("poisson7", 24, 2)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    xn, rn = solve(A, S["b"], s=12, basis="newton", tol=1e-8, maxit=300)
    assert rn.status == sscg.OK and rn.rel_res_true < 1e-7
    k = oracle.pcg(oracle.as_matrix(S), S["b"], tol=1e-8).iters
    assert rn.outer_iters <= -(-k // 12) + 1
    xm, rm = solve(A, S["b"], s=12, tol=1e-8, maxit=300)
    assert rm.status != sscg.OK or rm.outer_iters > rn.outer_iters


def test_adaptive_s_restarts_after_breakdown(ctx):
    """Monomial s = 16 breaks down (Section II-A's instability); with the
    adaptive block size the solve restarts from the last good iterate with s
    halved until it converges, and its solution matches the oracle's."""
    S = system("varcoef7", 12, 4, 1.0)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    x0, r0 = solve(A, S["b"], s=16, tol=1e-10, maxit=200)
    assert r0.status == sscg.BREAKDOWN and r0.profile["s_final"] == 16
    x, res = solve(A, S["b"], s=16, tol=1e-10, maxit=200, adaptive_s=True)
    assert res.status == sscg.OK and res.rel_res_true < 1e-9
    assert res.profile["s_final"] < 16
    assert len(res.hist) >= res.outer_iters  # segments' histories concatenated
    ref = oracle.pcg(oracle.as_matrix(S), S["b"], tol=1e-12, maxit=5000)
    assert rel(x, ref.x) < 1e-7
    # a solve that does not break down is untouched by the flag
    xa, ra = solve(A, S["b"], s=4, tol=1e-9, maxit=200, adaptive_s=True)
    xb, rb = solve(A, S["b"], s=4, tol=1e-9, maxit=200)
    assert ra.profile["s_final"] == 4 and ra.outer_iters == rb.outer_iters and np.array_equal(xa, xb)
