"""Parity of the CUDA s-step PCG and PCG (through the C ABI) with the FP64
CPU oracle.

Bars (from the solver's contract): at rel. residual tol, solution error vs
the oracle <= 1e-7 relative at the same outer-step count, outer-step counts
within +-1 of the oracle's, recursive residual below tol.  Iterates are
compared at equal step counts because both sides approximate the same
exact-arithmetic iterate x_{is}; a one-step difference in where a run stops
can move x by more than the bar on its own.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_03743_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_03743_gb300 import sscg  # noqa: E402

EPS = np.finfo(np.float64).eps


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


def gpu_matrix(ctx, sysm):
    return sscg.Matrix(ctx, sysm["rowptr"], sysm["col"], sysm["val"])


def gpu_solve(A, b, method="sstep", x0=None, **kw):
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    xt = torch.zeros_like(bt) if x0 is None else torch.from_numpy(np.array(x0, dtype=np.float64)).cuda()
    res = sscg.Solver(A, method=method, **kw).solve(bt, xt)
    return xt.cpu().numpy(), res


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SYSTEMS = [("poisson7", 19, 0, 0.0), ("varcoef7", 14, 1, 1.5), ("poisson27", 11, 2, 0.0)]


# ----------------------------------------------------------------- matrix

def test_matrix_properties(ctx):
    for kind, N, seed, sig in SYSTEMS:
        S = system(kind, N, seed, sig)
        A = gpu_matrix(ctx, S)
        p = A.props()
        rows = np.repeat(np.arange(S["n"]), np.diff(S["rowptr"]))
        assert p["n"] == S["n"] and p["nnz"] == len(S["col"])
        assert p["bandwidth"] == np.abs(S["col"] - rows).max()
        exact = bool(np.all(S["val"].astype(np.float32).astype(np.float64) == S["val"]))
        assert p["values_exact_fp32"] == int(exact)
        d = oracle.diag(oracle.as_matrix(S))
        assert p["diag_min"] == d.min() and p["diag_max"] == d.max()
        assert p["max_row_nnz"] == np.diff(S["rowptr"]).max()


def test_spmv_matches_oracle(ctx):
    for kind, N, seed, sig in SYSTEMS:
        S = system(kind, N, seed, sig)
        A = gpu_matrix(ctx, S)
        x = inputs.uniform(77, S["n"])
        y = A.spmv(torch.from_numpy(x).cuda()).cpu().numpy()
        yo = oracle.spmv(oracle.as_matrix(S), x)
        absAx = oracle.spmv(oracle.Matrix(S["rowptr"], S["col"], np.abs(S["val"])), np.abs(x))
        nnz_row = np.diff(S["rowptr"])
        assert np.all(np.abs(y - yo) <= 2 * nnz_row * EPS * absAx + 1e-300)


# ------------------------------------------------------------------- PCG

@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("case", range(len(SYSTEMS)))
def test_pcg_parity(ctx, arith, case):
    kind, N, seed, sig = SYSTEMS[case]
    S = system(kind, N, seed, sig)
    A = gpu_matrix(ctx, S)
    tol = 1e-8
    x, res = gpu_solve(A, S["b"], method="pcg", tol=tol, maxit=2000, arith=arith)
    assert res.status == sscg.OK
    assert res.rel_res_recursive < tol
    ref = oracle.pcg(oracle.as_matrix(S), S["b"], tol=tol, maxit=2000)
    assert abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pcg(oracle.as_matrix(S), S["b"], tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7
    assert res.rel_res_true < 2 * tol
    assert np.allclose(res.hist, same.hist, rtol=1e-5, atol=0)


# ---------------------------------------------------------------- s-step

@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("s", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("case", [0, 1])
def test_sstep_parity(ctx, arith, s, case):
    kind, N, seed, sig = SYSTEMS[case]
    S = system(kind, N, seed, sig)
    A = gpu_matrix(ctx, S)
    tol = 1e-8
    if arith == "df64" and s > 6:
        # the monomial basis at s = 8 amplifies rounding: FP64 on the GPU already
        # differs from the FP64 oracle by ~1.3e-8 there, and double-float's unit
        # roundoff (32x FP64's) would put it at ~1.1e-7, so the library refuses
        _expect_error(lambda: gpu_solve(A, S["b"], s=s, tol=tol, maxit=1000, arith=arith), sscg.ERR_INVALID)
        return
    x, res = gpu_solve(A, S["b"], s=s, tol=tol, maxit=1000, arith=arith)
    ref = oracle.pcgs(oracle.as_matrix(S), S["b"], s, tol=tol, maxit=1000)
    if ref.status == oracle.OK:
        assert res.status == sscg.OK, res
        assert res.rel_res_recursive < tol
        assert abs(res.outer_iters - ref.iters) <= 1
        same = oracle.pcgs(oracle.as_matrix(S), S["b"], s, tol=0.0, maxit=res.outer_iters)
        assert rel(x, same.x) < 1e-7, rel(x, same.x)
        assert res.rel_res_true < 10 * tol
    else:
        # monomial instability (Section II-A): the GPU must stop too and
        # leave a finite iterate
        assert res.status in (sscg.BREAKDOWN, sscg.NOT_CONVERGED)
        assert np.all(np.isfinite(x))


@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_config_32cubed_s4_beside_pcg(ctx, arith):
    """7-point 32^3, Jacobi, s = 4 monomial, b = A x_true, x0 = 0, tol 1e-8,
    checked against plain PCG and the oracle."""
    S = system("poisson7", 32, 0)
    A = gpu_matrix(ctx, S)
    x, res = gpu_solve(A, S["b"], s=4, tol=1e-8, maxit=500, arith=arith)
    xp, rp = gpu_solve(A, S["b"], method="pcg", tol=1e-8, maxit=2000, arith=arith)
    assert res.status == sscg.OK and rp.status == sscg.OK
    assert abs(res.equiv_iters - rp.outer_iters) <= 4
    ref = oracle.pcgs(oracle.as_matrix(S), S["b"], 4, tol=1e-8)
    assert abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pcgs(oracle.as_matrix(S), S["b"], 4, tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7
    assert rel(x, S["x_true"]) < 1e-5


def test_block_equivalence_on_gpu(ctx):
    """x_i of the s-step method equals PCG's x_{is} (Section II-A)."""
    S = system("varcoef7", 14, 1, 1.5)
    A = gpu_matrix(ctx, S)
    for s in (2, 4):
        for steps in (3, 7):
            xs, rs = gpu_solve(A, S["b"], s=s, tol=0.0, maxit=steps, arith="df64")
            xp, rp = gpu_solve(A, S["b"], method="pcg", tol=0.0, maxit=steps * s, arith="df64")
            assert rs.status == sscg.NOT_CONVERGED and rs.outer_iters == steps
            assert rp.outer_iters == steps * s
            assert rel(xs, xp) < 1e-9


# -------------------------------------------------------------- edge cases

def test_zero_rhs_gives_zero(ctx):
    S = system("poisson7", 9)
    A = gpu_matrix(ctx, S)
    for method in ("sstep", "pcg"):
        x, res = gpu_solve(A, np.zeros(S["n"]), method=method, x0=np.ones(S["n"]), tol=1e-8, maxit=50)
        assert res.status == sscg.OK and res.outer_iters == 0
        assert np.all(x == 0.0)


def test_exact_start_takes_no_step(ctx):
    S = system("poisson7", 9)
    A = gpu_matrix(ctx, S)
    for method in ("sstep", "pcg"):
        x, res = gpu_solve(A, S["b"], method=method, x0=S["x_true"], tol=1e-8, maxit=50)
        assert res.status == sscg.OK and res.outer_iters == 0
        assert np.array_equal(x, S["x_true"])


def test_maxit_zero_and_maxit_reached(ctx):
    S = system("poisson7", 12)
    A = gpu_matrix(ctx, S)
    x0 = inputs.uniform(3, S["n"])
    x, res = gpu_solve(A, S["b"], x0=x0, s=4, tol=1e-8, maxit=0)
    assert res.status == sscg.NOT_CONVERGED and res.outer_iters == 0
    assert np.array_equal(x, x0)
    x, res = gpu_solve(A, S["b"], s=4, tol=1e-14, maxit=3)
    assert res.status == sscg.NOT_CONVERGED and res.outer_iters == 3 and len(res.hist) == 4


@pytest.mark.parametrize("n", [1, 2, 5, 255, 256, 257, 1000])
def test_tiny_and_ragged_sizes(ctx, n):
    """Sizes around one 256-row tile, and 1 x 1."""
    rp, c, v = inputs.poisson7(max(1, round(n ** (1 / 3))))
    if len(rp) - 1 != n:  # ragged: a tridiagonal SPD matrix of exactly n rows
        rows = np.arange(n)
        cols = np.stack([rows - 1, rows, rows + 1], 1)
        vals = np.stack([-np.ones(n), 2.5 + np.abs(inputs.uniform(5, n)), -np.ones(n)], 1)
        ok = (cols >= 0) & (cols < n)
        rp = np.concatenate([[0], np.cumsum(ok.sum(1))]).astype(np.int32)
        c, v = cols[ok].astype(np.int32), vals[ok]
    S = dict(rowptr=rp, col=c, val=v)
    A = gpu_matrix(ctx, S)
    b = inputs.uniform(9, n)
    s = min(2, n)  # the Krylov space of an n x n system has dimension <= n
    for arith in ("f64", "df64"):
        x, res = gpu_solve(A, b, s=s, tol=1e-10, maxit=500, arith=arith)
        ref = oracle.pcgs(oracle.as_matrix(S), b, s, tol=1e-10, maxit=500)
        if ref.status == oracle.OK:
            assert res.status == sscg.OK
            assert abs(res.outer_iters - ref.iters) <= 1
            D = oracle.as_matrix(S).to_dense() if n <= 1000 else None
            assert rel(x, np.linalg.solve(D, b)) < 1e-8
        else:
            assert res.status != sscg.OK or res.outer_iters <= ref.iters + 1


def test_breakdown_is_reported_and_x_stays_finite(ctx):
    """Monomial s = 16 on a well-conditioned system loses independence."""
    S = system("varcoef7", 10, 4, 0.5)
    A = gpu_matrix(ctx, S)
    x, res = gpu_solve(A, S["b"], s=16, tol=1e-12, maxit=100)
    ref = oracle.pcgs(oracle.as_matrix(S), S["b"], 16, tol=1e-12, maxit=100)
    assert ref.status != oracle.OK
    assert res.status in (sscg.BREAKDOWN, sscg.NOT_CONVERGED)
    assert np.all(np.isfinite(x))


def test_host_vectors_path_matches_device_path(ctx):
    S = system("poisson7", 16, 3)
    A = gpu_matrix(ctx, S)
    xd, rd = gpu_solve(A, S["b"], s=4, tol=1e-8, maxit=200)
    xh = np.zeros(S["n"])
    rh = sscg.Solver(A, s=4, tol=1e-8, maxit=200, host_vectors=True).solve(np.ascontiguousarray(S["b"]), xh)
    assert rh.status == rd.status and rh.outer_iters == rd.outer_iters
    assert np.array_equal(xh, xd)


def _expect_error(fn, code):
    with pytest.raises(sscg.SscgError) as e:
        fn()
    assert e.value.code == code


def test_invalid_arguments(ctx):
    S = system("poisson7", 8)
    A = gpu_matrix(ctx, S)
    b = torch.from_numpy(S["b"]).cuda()
    for s in (0, 17):
        _expect_error(lambda: sscg.Solver(A, s=s), sscg.ERR_INVALID)
    _expect_error(lambda: sscg.Solver(A, s=4, maxit=-1), sscg.ERR_INVALID)
    sol = sscg.Solver(A, s=4, maxit=10)
    x = torch.zeros_like(b)
    small = sol.workspace[: sol.workspace.numel() // 2]
    sol.workspace, full = small, sol.workspace
    _expect_error(lambda: sol.solve(b, x), sscg.ERR_SPACE)
    sol.workspace = full[1:]  # misaligned
    _expect_error(lambda: sol.solve(b, x), sscg.ERR_SPACE)
    bn = b.clone()
    bn[3] = float("nan")
    sol.workspace = full
    _expect_error(lambda: sol.solve(bn, torch.zeros_like(b)), sscg.ERR_NONFINITE)


def test_matrix_rejections(ctx):
    S = system("poisson7", 6)
    v = S["val"].copy()
    v[S["rowptr"][5]:S["rowptr"][6]] = np.where(S["col"][S["rowptr"][5]:S["rowptr"][6]] == 5, -1.0,
                                                 v[S["rowptr"][5]:S["rowptr"][6]])
    _expect_error(lambda: sscg.Matrix(ctx, S["rowptr"], S["col"], v), sscg.ERR_NOT_SPD)
    c = S["col"].copy()
    c[10] = S["n"]
    _expect_error(lambda: sscg.Matrix(ctx, S["rowptr"], c, S["val"]), sscg.ERR_INVALID)
    v = S["val"].copy()
    v[7] = np.inf
    _expect_error(lambda: sscg.Matrix(ctx, S["rowptr"], S["col"], v), sscg.ERR_NONFINITE)
    rp = S["rowptr"].copy()
    rp[4], rp[5] = rp[5], rp[4]
    _expect_error(lambda: sscg.Matrix(ctx, rp, S["col"], S["val"]), sscg.ERR_INVALID)


@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_identity_preconditioner(ctx, arith):
    """B = I.  On the 7-point stencil D = 6 I, so B = I and Jacobi give the
    same iterates (the oracle pins that), and the GPU must match the
    oracle's B = I run."""
    S = system("poisson7", 13, 5)
    A = gpu_matrix(ctx, S)
    A.set_preconditioner("none")
    x, res = gpu_solve(A, S["b"], s=3, tol=1e-8, maxit=500, arith=arith)
    ref = oracle.pcgs(oracle.as_matrix(S), S["b"], 3, prec="none", tol=1e-8, maxit=500)
    assert ref.status == oracle.OK
    assert res.status == sscg.OK and abs(res.outer_iters - ref.iters) <= 1
    same = oracle.pcgs(oracle.as_matrix(S), S["b"], 3, prec="none", tol=0.0, maxit=res.outer_iters)
    assert rel(x, same.x) < 1e-7
    xj, rj = gpu_solve(gpu_matrix(ctx, S), S["b"], s=3, tol=1e-8, maxit=500, arith=arith)
    assert rj.outer_iters == res.outer_iters and rel(xj, x) < 1e-10


@pytest.mark.parametrize("s", [3, 4, 8])
def test_fused_mpk_matches_sequential_and_oracle(ctx, s):
    """128^3: large enough that the fused matrix-powers kernel runs (several
    levels per launch, levels kept in L2); it must give the sequential
    kernel's iterates and the oracle's."""
    S = system("poisson7", 128, 7)
    A = gpu_matrix(ctx, S)
    x, res = gpu_solve(A, S["b"], s=s, tol=1e-8, maxit=400, fused_mpk=True)
    xs, rs = gpu_solve(A, S["b"], s=s, tol=1e-8, maxit=400)
    assert res.status == rs.status
    assert res.outer_iters == rs.outer_iters
    # the two kernels accumulate the moments in different orders; the monomial
    # Hankel system amplifies that at s = 8 (Section II-A's instability)
    assert rel(x, xs) < (1e-9 if s <= 4 else 1e-5)
    if res.status == sscg.OK and s <= 4:
        ref = oracle.pcgs(oracle.as_matrix(S), S["b"], s, tol=0.0, maxit=res.outer_iters)
        assert rel(x, ref.x) < 1e-7
        assert res.rel_res_true < 1e-7


# ------------------------------------------------------------- full size

@pytest.mark.slow
@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_full_size_256_s4_against_oracle(ctx, arith):
    """7-point 256^3, Jacobi, s = 4, tol 1e-8, in the launch configuration
    the benchmark times, against the oracle run to the same outer step."""
    S = system("poisson7", 256, 0)
    A = gpu_matrix(ctx, S)
    x, res = gpu_solve(A, S["b"], s=4, tol=1e-8, maxit=2000, arith=arith)
    assert res.status == sscg.OK and res.rel_res_recursive < 1e-8 and res.rel_res_true < 2e-8
    M = oracle.as_matrix(S)
    if "ref256" not in _CACHE:  # the same oracle run serves both arithmetics
        _CACHE["ref256"] = oracle.pcgs(M, S["b"], 4, tol=1e-8, maxit=2000)
    ref = _CACHE["ref256"]
    assert ref.status == oracle.OK and abs(res.outer_iters - ref.iters) <= 1
    if ref.iters != res.outer_iters:
        ref = oracle.pcgs(M, S["b"], 4, tol=0.0, maxit=res.outer_iters)
    assert rel(x, ref.x) < 1e-7


# ------------------------------------------------------- diagonal form

def test_diagonal_form_detection(ctx):
    """Constant stencils are multiplied in the diagonal form; variable
    coefficients, a perturbed stencil and CSR-only creation stay CSR."""
    for kind, N, want in (("poisson7", 9, 7), ("poisson27", 7, 27), ("aniso7", 9, 7)):
        S = system(kind, N, 0)
        assert gpu_matrix(ctx, S).props()["format"] == 1
        assert gpu_matrix(ctx, S).props()["dia_offsets"] == want
        assert sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"], csr_only=True).props()["format"] == 0
    assert gpu_matrix(ctx, system("varcoef7", 9, 0, 1.0)).props()["format"] == 0
    S = system("poisson7", 6, 0)
    val = S["val"].copy()
    val[100] *= 1.0 + 2.0 ** -40  # one value off the stencil (and not FP32-exact)
    assert sscg.Matrix(ctx, S["rowptr"], S["col"], val).props()["format"] == 0
    val = S["val"].copy()
    val[100] = -2.0  # FP32-exact, but not the diagonal's constant
    assert sscg.Matrix(ctx, S["rowptr"], S["col"], val).props()["format"] == 0


@pytest.mark.parametrize("arith", ["f64", "df64"])
@pytest.mark.parametrize("kind,N", [("poisson7", 21), ("poisson27", 13), ("aniso7", 17), ("poisson7", 16)])
def test_diagonal_form_matches_csr_and_oracle(ctx, arith, kind, N):
    S = system(kind, N, 3)
    Ad = gpu_matrix(ctx, S)
    Ac = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"], csr_only=True)
    assert Ad.props()["format"] == 1 and Ac.props()["format"] == 0
    for method, s in (("sstep", 4), ("sstep", 2), ("pcg", 1)):
        xd, rd = gpu_solve(Ad, S["b"], method=method, s=s, tol=1e-9, maxit=2000, arith=arith)
        xc, rc = gpu_solve(Ac, S["b"], method=method, s=s, tol=1e-9, maxit=2000, arith=arith)
        assert rd.status == rc.status == sscg.OK
        assert rd.outer_iters == rc.outer_iters
        assert rel(xd, xc) < 1e-11
    ref = oracle.pcgs(oracle.as_matrix(S), S["b"], 4, tol=1e-9, maxit=2000)
    xd, rd = gpu_solve(Ad, S["b"], s=4, tol=1e-9, maxit=2000, arith=arith)
    assert abs(rd.outer_iters - ref.iters) <= 1
    same = oracle.pcgs(oracle.as_matrix(S), S["b"], 4, tol=0.0, maxit=rd.outer_iters)
    assert rel(xd, same.x) < 1e-7


@pytest.mark.parametrize("kind,N", [("poisson7", 19), ("aniso7", 15), ("poisson27", 11), ("poisson7", 12)])
def test_diagonal_form_in_gram_and_mixed_paths(ctx, kind, N):
    """The direct-Gram levels (Chebyshev and monomial bases) and the
    mixed-precision levels and residual replacement multiply in the diagonal
    form; each matches the same solve on the CSR arrays (odd and even n,
    the Laplacian class and a stencil with unequal couplings)."""
    S = system(kind, N, 5)
    Ad = gpu_matrix(ctx, S)
    Ac = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"], csr_only=True)
    assert Ad.props()["format"] == 1 and Ac.props()["format"] == 0
    cases = (
        dict(s=6, basis="chebyshev", tol=1e-9, maxit=2000, arith="df64", basis_bounds=(0.05, 2.0)),
        dict(s=4, tol=1e-9, maxit=2000, arith="df64", direct_gram=True),
        dict(s=4, tol=1e-9, maxit=2000, arith="mixed", replace_every=1),
        dict(s=4, basis="chebyshev", tol=1e-9, maxit=2000, arith="mixed", replace_every=2,
             basis_bounds=(0.05, 2.0)),
    )
    for kw in cases:
        xd, rd = gpu_solve(Ad, S["b"], **kw)
        xc, rc = gpu_solve(Ac, S["b"], **kw)
        assert rd.status == rc.status == sscg.OK, kw
        assert abs(rd.outer_iters - rc.outer_iters) <= (1 if kw["arith"] == "mixed" else 0), kw
        # mixed: the FP32 basis rounds differently when A u is summed in another order
        assert rel(xd, xc) < (1e-6 if kw["arith"] == "mixed" else 1e-10), kw
        assert rel(xd, S["x_true"]) < 1e-6, kw


# ------------------------------------------------- double-float range

def test_df64_refuses_right_hand_sides_outside_fp32_range(ctx):
    """A double-float solve carries its vectors and squared norms in FP32's
    exponent range: b scaled by 1e-25 would underflow ||b||^2 (a silent x = 0
    before) and is refused; the FP64 solve of the same system is the scaled
    solution."""
    S = system("poisson7", 12, 1)
    A = gpu_matrix(ctx, S)
    x1, r1 = gpu_solve(A, S["b"], s=4, tol=1e-9, maxit=300, arith="f64")
    for scale in (1e-25, 1e25):
        bs = S["b"] * scale
        for method in ("sstep", "pcg"):
            _expect_error(lambda: gpu_solve(A, bs, method=method, s=4, tol=1e-9, maxit=300, arith="df64"),
                          sscg.ERR_INVALID)
        xs, rs = gpu_solve(A, bs, s=4, tol=1e-9, maxit=300, arith="f64")
        assert rs.status == sscg.OK and rs.outer_iters == r1.outer_iters
        assert rel(xs / scale, x1) < 1e-12


def test_df64_refuses_matrix_values_outside_fp32_range(ctx):
    """Values below FP32's normal range (1e-40 on the diagonal) flush to zero
    in double-float: df64 solves refuse such a matrix, f64 solves it."""
    n = 64
    rp = np.arange(n + 1, dtype=np.int32)
    c = np.arange(n, dtype=np.int32)
    v = np.full(n, 1e-40)
    A = sscg.Matrix(ctx, rp, c, v)
    b = inputs.uniform(4, n)
    for method in ("sstep", "pcg"):
        _expect_error(lambda: gpu_solve(A, b, method=method, s=1, tol=1e-10, maxit=10, arith="df64"),
                      sscg.ERR_INVALID)
    x, res = gpu_solve(A, b, s=1, tol=1e-10, maxit=10, arith="f64")  # D^-1 A = I: one step
    assert res.status == sscg.OK and rel(x, b / 1e-40) < 1e-14
