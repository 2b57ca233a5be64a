"""The batched persistent solver through the C ABI: every right-hand side of
every system against the FP64 oracle (same outer-step count, x to 1e-7),
against the single-system solver, edge cases, the autotuner and argument
checks."""
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


def random_spd(n, seed):
    u = inputs.uniform(seed, n * n).reshape(n, n)
    S = np.triu(np.where(np.abs(u) < 0.3, u, 0.0), 1)
    S = S + S.T
    D = S + np.diag(np.abs(S).sum(1) + 0.5 + np.abs(inputs.uniform(seed + 1, n)))
    M = oracle.Matrix.from_dense(D)
    return M.rowptr, M.col, M.val


def csr(kind, N, seed=0, sigma=1.0):
    if kind == "varcoef7":
        return inputs.varcoef7(N, sigma, seed, 4.0)
    if kind == "dense":
        return random_spd(N, seed)
    return getattr(inputs, kind)(N)


# (kind, size, seed, nrhs): exact FP32 values (stencils) and inexact ones
# (variable coefficients, random dense), tiles shorter than one item, ragged
# tails, 1..8 right-hand sides.
MIX = [("poisson7", 6, 0, 1), ("poisson7", 13, 0, 3), ("poisson27", 7, 0, 2), ("varcoef7", 10, 5, 8),
       ("dense", 40, 7, 5), ("varcoef7", 17, 6, 4), ("poisson7", 24, 0, 2), ("dense", 9, 9, 1)]


def make_batch(ctx, spec, rhs_seed=100):
    mats, csrs, B, X = [], [], [], []
    for i, (kind, N, seed, R) in enumerate(spec):
        c = csr(kind, N, seed)
        csrs.append(c)
        A = sscg.Matrix(ctx, *c)
        mats.append(A)
        n = A.n
        xt = inputs.uniform(rhs_seed + i, R * n).reshape(R, n)
        b = np.stack([inputs.matvec(*c, xt[r]) for r in range(R)])
        B.append(torch.from_numpy(b).cuda())
        X.append(torch.zeros(R, n, dtype=torch.float64, device="cuda"))
    return mats, csrs, B, X


@pytest.mark.parametrize("persistent", [False, True], ids=["phases", "persistent"])
@pytest.mark.parametrize("arith", ["df64", "f64"])
@pytest.mark.parametrize("s", [2, 4])
def test_batch_matches_oracle_per_rhs(ctx, arith, s, persistent):
    mats, csrs, B, X = make_batch(ctx, MIX)
    plan = sscg.BatchSolver(mats, [m[3] for m in MIX], s=s, tol=1e-8, maxit=500, arith=arith, persistent=persistent)
    res = plan.solve(B, X)
    assert res.status == sscg.OK
    q = 0
    for i, (spec, c) in enumerate(zip(MIX, csrs)):
        M = oracle.Matrix(*c)
        b = B[i].cpu().numpy()
        x = X[i].cpu().numpy()
        worst = 0
        for r in range(spec[3]):
            info = res.rhs[q]
            q += 1
            ref = oracle.pcgs(M, b[r], s, tol=1e-8, maxit=500)
            assert ref.status == oracle.OK
            assert info.status == sscg.OK and info.rel_res_recursive < 1e-8
            assert abs(info.outer_iters - ref.iters) <= 1, (spec, r, info.outer_iters, ref.iters)
            same = oracle.pcgs(M, b[r], s, tol=0.0, maxit=info.outer_iters)
            assert rel(x[r], same.x) < 1e-7, (spec, r)
            assert info.rel_res_true < 1e-7
            worst = max(worst, info.outer_iters)
        assert res.systems[i].outer_iters == worst
    assert np.all(res.latency_ms > 0) and np.all(res.latency_ms <= res.solve_ms * 1.01 + 0.05)


@pytest.mark.parametrize("persistent", [False, True], ids=["phases", "persistent"])
def test_batch_matches_single_system_solver(ctx, persistent):
    spec = [("varcoef7", 16, 3, 3), ("poisson27", 9, 0, 1), ("poisson7", 20, 0, 2)]
    mats, csrs, B, X = make_batch(ctx, spec, rhs_seed=7)
    res = sscg.BatchSolver(mats, [m[3] for m in spec], s=4, tol=1e-9, maxit=400, persistent=persistent).solve(B, X)
    q = 0
    for i, (sp, A) in enumerate(zip(spec, mats)):
        for r in range(sp[3]):
            x1 = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            r1 = sscg.Solver(A, s=4, tol=1e-9, maxit=400).solve(B[i][r].contiguous(), x1)
            assert r1.outer_iters == res.rhs[q].outer_iters
            assert rel(X[i][r].cpu().numpy(), x1.cpu().numpy()) < 1e-10
            q += 1


def test_batch_edge_cases(ctx):
    """Nonzero x0, a zero right-hand side and an exact start in one system,
    beside a plain one: each is reported per right-hand side."""
    cp = csr("poisson7", 9)
    A1, A2 = sscg.Matrix(ctx, *cp), sscg.Matrix(ctx, *cp)
    n = A1.n
    xt = inputs.uniform(1, 3 * n).reshape(3, n)
    b1 = np.stack([inputs.matvec(*cp, xt[0]), np.zeros(n), inputs.matvec(*cp, xt[2])])
    x01 = np.stack([inputs.uniform(2, n), inputs.uniform(3, n), xt[2]])  # the last x0 is exact
    b2 = inputs.matvec(*cp, inputs.uniform(4, n))[None, :]
    B = [torch.from_numpy(b1).cuda(), torch.from_numpy(b2).cuda()]
    X = [torch.from_numpy(x01.copy()).cuda(), torch.zeros(1, n, dtype=torch.float64, device="cuda")]
    res = sscg.BatchSolver([A1, A2], [3, 1], s=4, tol=1e-10, maxit=200).solve(B, X)
    assert res.status == sscg.OK
    x = X[0].cpu().numpy()
    assert res.rhs[0].status == sscg.OK and rel(x[0], xt[0]) < 1e-8
    assert res.rhs[1].outer_iters == 0 and np.all(x[1] == 0.0)
    assert res.rhs[2].outer_iters == 0 and np.array_equal(x[2], xt[2])
    ref = oracle.pcgs(oracle.Matrix(*cp), b2[0], 4, tol=1e-10, maxit=200)
    assert abs(res.rhs[3].outer_iters - ref.iters) <= 1


def test_batch_failure_stays_local(ctx):
    """A right-hand side with a NaN entry fails alone: it is reported as a
    breakdown (non-finite value) with x left finite, and the other system's
    outcome is the one the single-system solver gets."""
    cv = csr("varcoef7", 10, 4, 0.5)
    cp = csr("poisson7", 7)
    Av, Ap = sscg.Matrix(ctx, *cv), sscg.Matrix(ctx, *cp)
    bv = np.stack([inputs.matvec(*cv, inputs.uniform(5, Av.n)), inputs.matvec(*cv, inputs.uniform(7, Av.n))])
    bv[0, 17] = np.nan
    bp = inputs.matvec(*cp, inputs.uniform(6, Ap.n))[None, :]
    B = [torch.from_numpy(bv).cuda(), torch.from_numpy(bp).cuda()]
    X = [torch.zeros_like(B[0]), torch.zeros_like(B[1])]
    res = sscg.BatchSolver([Av, Ap], [2, 1], s=4, tol=1e-9, maxit=300).solve(B, X)
    assert res.status == sscg.BREAKDOWN
    assert res.rhs[0].status == sscg.BREAKDOWN and res.rhs[0].outer_iters == 0
    assert res.rhs[1].status == sscg.OK and res.rhs[1].rel_res_true < 1e-8
    assert np.all(np.isfinite(X[0].cpu().numpy())) and np.all(np.isfinite(X[1].cpu().numpy()))
    x1 = torch.zeros(Ap.n, dtype=torch.float64, device="cuda")
    single = sscg.Solver(Ap, s=4, tol=1e-9, maxit=300).solve(B[1][0].contiguous(), x1)
    assert res.rhs[2].status == single.status and res.rhs[2].outer_iters == single.outer_iters
    assert rel(X[1][0].cpu().numpy(), x1.cpu().numpy()) < 1e-10


def test_batch_maxit_reached(ctx):
    c = csr("poisson7", 12)
    A = sscg.Matrix(ctx, *c)
    b = torch.from_numpy(inputs.matvec(*c, inputs.uniform(3, A.n))[None, :]).cuda()
    x = torch.zeros_like(b)
    res = sscg.BatchSolver([A], [1], s=2, tol=1e-10, maxit=3).solve([b], [x])
    assert res.status == sscg.NOT_CONVERGED and res.rhs[0].outer_iters == 3
    same = oracle.pcgs(oracle.Matrix(*c), b[0].cpu().numpy(), 2, tol=0.0, maxit=3)
    assert rel(x[0].cpu().numpy(), same.x) < 1e-9


def test_autotuned_plan_agrees(ctx):
    spec = [("poisson7", 40, 0, 2), ("varcoef7", 24, 2, 3), ("poisson27", 30, 0, 1), ("poisson7", 70, 0, 1)]
    mats, csrs, B, X = make_batch(ctx, spec, rhs_seed=11)
    fixed = sscg.BatchSolver(mats, [m[3] for m in spec], s=4, tol=1e-8, maxit=600)
    tuned = sscg.BatchSolver(mats, [m[3] for m in spec], s=4, tol=1e-8, maxit=600, tune=True)
    tiles = tuned.props()["tile_rows"]
    assert all(t in (256, 512, 1024, 2048, 4096) for t in tiles)
    # systems of one size class share a tile
    assert tiles[0] == tiles[1] or (mats[0].n >= 1 << 16) != (mats[1].n >= 1 << 16)
    r1 = fixed.solve(B, X)
    X2 = [torch.zeros_like(x) for x in X]
    r2 = tuned.solve(B, X2)
    assert r1.status == r2.status == sscg.OK
    for a, b in zip(r1.rhs, r2.rhs):
        assert abs(a.outer_iters - b.outer_iters) <= 1
    for xa, xb in zip(X, X2):
        assert rel(xb.cpu().numpy(), xa.cpu().numpy()) < 1e-8


def test_batch_latency_orders_sizes(ctx):
    """A small system's result is final well before a large one's."""
    spec = [("poisson7", 8, 0, 1), ("poisson7", 64, 0, 1)]
    mats, csrs, B, X = make_batch(ctx, spec)
    res = sscg.BatchSolver(mats, [1, 1], s=4, tol=1e-8, maxit=500).solve(B, X)
    assert res.status == sscg.OK
    assert res.latency_ms[0] < 0.5 * res.latency_ms[1]


def test_batch_invalid_arguments(ctx):
    c = csr("poisson7", 6)
    A = sscg.Matrix(ctx, *c)
    for kw in (dict(s=9), dict(s=0), dict(arith="mixed")):
        with pytest.raises(sscg.SscgError):
            sscg.BatchSolver([A], [1], **kw)
    with pytest.raises(sscg.SscgError):
        sscg.BatchSolver([A], [9])
    with pytest.raises(sscg.SscgError):
        sscg.BatchSolver([A], [0])
    lo, hi = inputs.closed_form_bounds("poisson7", 6)
    A.set_preconditioner("cheb", 2, lo / 6, hi / 6)
    with pytest.raises(sscg.SscgError):
        sscg.BatchSolver([A], [1])
    A.set_preconditioner("jacobi")
    opts = sscg.make_opts(s=4, basis="chebyshev", basis_bounds=(0.1, 2.0))
    import ctypes as C
    nb = C.c_size_t()
    mh = (C.c_void_p * 1)(A.h.value)
    nr = (C.c_int * 1)(1)
    assert ctx.lib.sscg_batch_workspace_bytes(1, mh, nr, C.byref(opts), C.byref(nb)) == sscg.ERR_INVALID
    ok = sscg.make_opts(s=4)
    assert ctx.lib.sscg_batch_workspace_bytes(1, mh, nr, C.byref(ok), C.byref(nb)) == sscg.OK
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    rc = ctx.lib.sscg_batch_create(ctx.h, 1, mh, nr, C.byref(ok), 0, C.c_void_p(ws.data_ptr()), nb.value - 256,
                                   C.byref(h))
    assert rc == sscg.ERR_SPACE


def test_bounded_barrier_wait_runs_out(ctx):
    """Failure detection without a GPU fault: one CTA of the persistent
    solve's cooperative launch skips its first grid-barrier arrival, so every
    other CTA's bounded wait (200 ms here) runs out.  The solve must come
    back with SSCG_TIMEOUT well inside a second, and the same plan's next
    solve must succeed and agree with a clean solve."""
    import time

    spec = [("poisson7", 12, 0, 2), ("varcoef7", 10, 3, 1)]
    mats, csrs, B, X = make_batch(ctx, spec, rhs_seed=31)
    plan = sscg.BatchSolver(mats, [m[3] for m in spec], s=4, tol=1e-9, maxit=300, persistent=True)
    grid = plan.props()["grid"]
    for x in X:
        x.zero_()
    ref = plan.solve(B, X)
    assert ref.status == sscg.OK
    x_ref = [x.clone() for x in X]
    for cta in (0, grid - 1):
        plan.inject_barrier_fault(cta, 200)
        for x in X:
            x.zero_()
        t0 = time.perf_counter()
        bad = plan.solve(B, X)
        assert bad.status == sscg.TIMEOUT
        assert time.perf_counter() - t0 < 5.0
        for x in X:
            x.zero_()
        again = plan.solve(B, X)  # disarmed: the plan and the context are still usable
        assert again.status == sscg.OK
        for x, xr in zip(X, x_ref):
            assert torch.equal(x, xr)
    with pytest.raises(sscg.SscgError):
        plan.inject_barrier_fault(grid, 200)
    with pytest.raises(sscg.SscgError):
        sscg.BatchSolver(mats, [m[3] for m in spec], s=4, tol=1e-9, maxit=300).inject_barrier_fault(0, 200)
