"""The FP64 block update with P and Q formed as fixed-point dot products on
the integer multipliers (the default at s <= 6) against the FP64 FMA update
(SSCG_FMA_UPDATE) and the FP64 oracle: the same outer-step counts (+-1),
solutions within 1e-9 of each other and within 1e-7 of the oracle at equal
step counts; rows whose values are all zero or below 2^-961 take the FP64 FMAs;
block sizes above 6 are untouched by the flag."""
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


CASES = [("poisson7", 19, 0, 0.0, False), ("varcoef7", 14, 1, 1.5, False), ("poisson27", 11, 2, 0.0, False),
         ("aniso7", 15, 3, 0.0, False), ("poisson7", 17, 4, 0.0, True)]


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_fixed_point_update_matches_fma_update_and_oracle(ctx, s, case):
    kind, N, seed, sig, csr = CASES[case]
    S = system(kind, N, seed, sig)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"], csr_only=csr)
    xf, rf = solve(A, S["b"], s=s, tol=1e-8, maxit=1000)
    xm, rm = solve(A, S["b"], s=s, tol=1e-8, maxit=1000, fma_update=True)
    assert rf.status == rm.status == sscg.OK
    assert abs(rf.outer_iters - rm.outer_iters) <= 1
    assert rf.rel_res_recursive < 1e-8 and rf.rel_res_true < 1e-7
    if rf.outer_iters == rm.outer_iters:
        assert rel(xf, xm) < 1e-9, rel(xf, xm)
        hf, hm = np.array(rf.hist), np.array(rm.hist)
        assert np.allclose(hf, hm, rtol=1e-6, atol=0)
    same = oracle.pcgs(oracle.as_matrix(S), S["b"], s, tol=0.0, maxit=rf.outer_iters)
    assert rel(xf, same.x) < 1e-7


def test_fixed_point_update_runs_and_differs_in_rounding(ctx):
    """The default s = 4 solve does not repeat the FMA update bit for bit (its
    dot products round once, the FMA chain s times), while s = 8 (above the
    fixed-point limit of s = 6) is identical with and without the flag."""
    S = system("poisson7", 19, 0)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    xf, rf = solve(A, S["b"], s=4, tol=1e-10, maxit=1000)
    xm, rm = solve(A, S["b"], s=4, tol=1e-10, maxit=1000, fma_update=True)
    assert not np.array_equal(xf, xm) and rel(xf, xm) < 1e-9
    x8, r8 = solve(A, S["b"], s=8, tol=1e-8, maxit=1000)
    y8, q8 = solve(A, S["b"], s=8, tol=1e-8, maxit=1000, fma_update=True)
    assert np.array_equal(x8, y8) and r8.outer_iters == q8.outer_iters


def test_rows_of_zeros_and_tiny_values_take_the_fma_path(ctx):
    """A right-hand side that is 1 on a corner block, about 1e-295 on a slab
    and 0 elsewhere: in the first outer steps most rows of U, P and Q are all
    zero or below 2^-961 and take the FP64 FMAs, the rest the fixed-point dot
    products, within the same warps.  Both updates agree and match the oracle."""
    N = 20
    S = system("poisson7", N, 6)
    rng = np.random.default_rng(6)
    b = np.zeros((N, N, N))
    b[:3, :3, :3] = rng.uniform(0.5, 1.0, (3, 3, 3))
    b[10:13] = rng.uniform(-1, 1, (3, N, N)) * 1e-295
    b = b.ravel()
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    xf, rf = solve(A, b, s=4, tol=1e-8, maxit=1000)
    xm, rm = solve(A, b, s=4, tol=1e-8, maxit=1000, fma_update=True)
    assert rf.status == rm.status == sscg.OK and abs(rf.outer_iters - rm.outer_iters) <= 1
    if rf.outer_iters == rm.outer_iters:
        assert rel(xf, xm) < 1e-9
    ref = oracle.pcgs(oracle.as_matrix(S), b, 4, tol=1e-8, maxit=1000)
    assert ref.status == oracle.OK and abs(rf.outer_iters - ref.iters) <= 1
    same = oracle.pcgs(oracle.as_matrix(S), b, 4, tol=0.0, maxit=rf.outer_iters)
    assert rel(xf, same.x) < 1e-7


@pytest.mark.parametrize("kind,N,sigma", [("poisson7", 32, 0.0), ("varcoef7", 24, 3.0), ("poisson27", 40, 0.0)])
def test_attainable_accuracy_matches_fma_update(ctx, kind, N, sigma):
    """Solved to 1e-12, where the gap between the recursive and the true
    residual shows how rounding in the updates accumulates: the fixed-point
    update's true residual is no larger than twice the FMA update's, and both
    solutions agree with the oracle's at equal step counts."""
    S = system(kind, N, 7, sigma)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    xf, rf = solve(A, S["b"], s=4, tol=1e-12, maxit=3000)
    xm, rm = solve(A, S["b"], s=4, tol=1e-12, maxit=3000, fma_update=True)
    assert rf.status == rm.status == sscg.OK
    assert rf.rel_res_true <= 2 * max(rm.rel_res_true, 1e-13), (rf.rel_res_true, rm.rel_res_true)
    same = oracle.pcgs(oracle.as_matrix(S), S["b"], 4, tol=0.0, maxit=rf.outer_iters)
    assert rel(xf, same.x) < 1e-7


def tridiagonal(n, seed):
    """SPD tridiagonal CSR: -1 off the diagonal, 4 + |u_i| on it (u seeded uniform)."""
    d = 4.0 + np.abs(inputs.uniform(seed, n))
    rows = np.arange(n)
    cols = np.stack([rows - 1, rows, rows + 1], axis=1)
    vals = np.stack([-np.ones(n), d, -np.ones(n)], axis=1)
    keep = (cols >= 0) & (cols < n)
    rowptr = np.concatenate([[0], np.cumsum(keep.sum(1))]).astype(np.int32)
    return dict(rowptr=rowptr, col=cols[keep].astype(np.int32), val=vals[keep])


@pytest.mark.parametrize("s", [2, 4, 6])
@pytest.mark.parametrize("mult,extra", [(1, 1), (2, -1), (3, 5)])
def test_update_row_prefetch_at_grid_stride_boundaries(ctx, s, mult, extra):
    """Each thread of the fixed-point update copies its next row (i + the grid's
    threads) to shared memory while it computes row i.  Row counts just above,
    just below and past multiples of the grid's threads at two CTAs per SM
    (s = 4, 6; s = 2 runs more CTAs) leave threads with different row counts,
    the last row of each taking the no-prefetch branch: the solution matches
    the FMA update's and the oracle's at equal step counts."""
    stride = torch.cuda.get_device_properties(0).multi_processor_count * 2 * 256
    n = mult * stride + extra
    S = tridiagonal(n, 11 + mult)
    b = inputs.uniform(40 + mult, n)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    xf, rf = solve(A, b, s=s, tol=1e-10, maxit=200)
    xm, rm = solve(A, b, s=s, tol=1e-10, maxit=200, fma_update=True)
    assert rf.status == rm.status == sscg.OK and abs(rf.outer_iters - rm.outer_iters) <= 1
    assert rf.outer_iters >= 2  # the fixed-point update runs from the second step on
    if rf.outer_iters == rm.outer_iters:
        assert rel(xf, xm) < 1e-9, rel(xf, xm)
    same = oracle.pcgs(oracle.as_matrix(S), b, s, tol=0.0, maxit=rf.outer_iters)
    assert rel(xf, same.x) < 1e-7
    assert rf.rel_res_true < 1e-9
