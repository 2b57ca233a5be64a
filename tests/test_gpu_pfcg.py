"""PFCG-NN (Algorithm 2) on the GPU through the C ABI against the FP64 CPU
oracle's Algorithm 2: iteration counts within +-1, x within 1e-7 at the same
iteration count, the residual history, the diagonal form against CSR, and
the edge cases."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def solve(A, b, x0=None, **kw):
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.zeros_like(bt) if x0 is None else torch.from_numpy(np.array(x0, dtype=np.float64)).cuda()
    res = sscg.Solver(A, method="pfcg", **kw).solve(bt, xt)
    return xt.cpu().numpy(), res


SYSTEMS = [("poisson7", 19, 0, 0.0), ("varcoef7", 14, 1, 1.5), ("poisson27", 11, 2, 0.0), ("aniso7", 15, 3, 0.0)]


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("case", range(len(SYSTEMS)))
def test_pfcg_parity(ctx, arith, case):
    kind, N, seed, sig = SYSTEMS[case]
    S = inputs.system(kind, N, seed=seed, sigma=sig)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    tol = 1e-8
    x, res = solve(A, S["b"], tol=tol, maxit=3000, arith=arith)
    assert res.status == sscg.OK
    assert res.rel_res_recursive < tol and res.rel_res_true < 2 * tol
    M = oracle.as_matrix(S)
    ref = oracle.pfcg(M, S["b"], tol=tol, maxit=3000)
    assert ref.status == oracle.OK and abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pfcg(M, S["b"], tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7
    assert np.allclose(res.hist, same.hist, rtol=1e-5, atol=0)


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("kind,N", [("poisson7", 21), ("poisson27", 13), ("aniso7", 16)])
def test_pfcg_diagonal_form_matches_csr(ctx, arith, kind, N):
    S = inputs.system(kind, N, seed=4)
    Ad = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    Ac = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"], csr_only=True)
    assert Ad.props()["format"] == 1 and Ac.props()["format"] == 0
    xd, rd = solve(Ad, S["b"], tol=1e-9, maxit=3000, arith=arith)
    xc, rc = solve(Ac, S["b"], tol=1e-9, maxit=3000, arith=arith)
    assert rd.status == rc.status == sscg.OK and rd.outer_iters == rc.outer_iters
    assert rel(xd, xc) < 1e-11


def test_pfcg_equals_pcg_for_a_fixed_preconditioner(ctx):
    """With a fixed B, Algorithm 2 generates the iterates of Algorithm 1."""
    S = inputs.system("varcoef7", 16, seed=6, sigma=1.0)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    bt = torch.from_numpy(S["b"]).cuda()
    for steps in (5, 40):
        xf, rf = solve(A, S["b"], tol=0.0, maxit=steps)
        xp = torch.zeros_like(bt)
        rp = sscg.Solver(A, method="pcg", tol=0.0, maxit=steps).solve(bt, xp)
        assert rf.outer_iters == rp.outer_iters == steps
        assert rel(xf, xp.cpu().numpy()) < 1e-10


def test_pfcg_identity_preconditioner_and_x0(ctx):
    S = inputs.system("poisson7", 12, seed=2)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    A.set_preconditioner("none")
    x0 = inputs.uniform(8, S["n"])
    x, res = solve(A, S["b"], x0=x0, tol=1e-9, maxit=2000)
    ref = oracle.pfcg(oracle.as_matrix(S), S["b"], x0=x0, prec="none", tol=1e-9, maxit=2000)
    assert res.status == sscg.OK and abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pfcg(oracle.as_matrix(S), S["b"], x0=x0, prec="none", tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7


def test_pfcg_edge_cases(ctx):
    S = inputs.system("poisson7", 9, seed=0)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    x, res = solve(A, np.zeros(S["n"]), x0=np.ones(S["n"]), tol=1e-8, maxit=50)
    assert res.status == sscg.OK and res.outer_iters == 0 and np.all(x == 0.0)
    x, res = solve(A, S["b"], x0=S["x_true"], tol=1e-8, maxit=50)
    assert res.status == sscg.OK and res.outer_iters == 0 and np.array_equal(x, S["x_true"])
    x0 = inputs.uniform(3, S["n"])
    x, res = solve(A, S["b"], x0=x0, tol=1e-8, maxit=0)
    assert res.status == sscg.NOT_CONVERGED and res.outer_iters == 0 and np.array_equal(x, x0)
    x, res = solve(A, S["b"], tol=1e-14, maxit=3)
    assert res.status == sscg.NOT_CONVERGED and res.outer_iters == 3 and len(res.hist) == 4
    bn = S["b"].copy()
    bn[5] = np.nan
    with pytest.raises(sscg.SscgError) as e:
        solve(A, bn, tol=1e-8, maxit=50)
    assert e.value.code == sscg.ERR_NONFINITE
    A.set_preconditioner("cheb", degree=2, lmin=0.1, lmax=2.0)
    with pytest.raises(sscg.SscgError) as e:
        solve(A, S["b"], tol=1e-8, maxit=50)
    assert e.value.code == sscg.ERR_INVALID
