"""sscg_solve_static, the solve for callers that cannot allocate device
memory (it takes its workspace from a fixed array inside the library), must
give the same answer as sscg_solve with caller workspace, on consecutive
calls that share that array.  This file is collected last so a run that stops
at the first failure has run every other test first; it also passes alone."""
import ctypes as C

import numpy as np
import pytest

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


def _static_solve(ctx, A, b, opts):
    x = torch.zeros_like(b)
    info = sscg.Info()
    rc = ctx.lib.sscg_solve_static(ctx.h, A.h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(opts),
                                   C.byref(info))
    torch.cuda.synchronize()
    return rc, x.cpu().numpy(), info


@pytest.mark.parametrize("kind,N,s,basis", [("poisson7", 30, 4, "monomial"), ("varcoef7", 24, 8, "chebyshev")])
def test_static_scratch_matches_caller_workspace(ctx, kind, N, s, basis):
    S = inputs.system(kind, N, seed=11, sigma=1.0)
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    b = torch.from_numpy(S["b"]).cuda()
    kw = dict(s=s, basis=basis, tol=1e-8, maxit=400)
    ref_x = torch.zeros_like(b)
    ref = sscg.Solver(A, **kw).solve(b, ref_x)
    ref_x = ref_x.cpu().numpy()
    assert ref.status == sscg.OK
    opts = sscg.make_opts(**kw)
    for _ in range(2):  # two calls in a row share the static array
        rc, x, info = _static_solve(ctx, A, b, opts)
        assert rc == sscg.OK, ctx.lib.sscg_last_error(ctx.h).decode()
        assert info.outer_iters == ref.outer_iters
        assert np.linalg.norm(x - ref_x) / np.linalg.norm(ref_x) < 1e-7
        assert info.rel_res_true < 1e-7


def test_static_scratch_rejects_oversize(ctx):
    S = inputs.system("poisson7", 64, seed=1)  # n = 262,144: workspace beyond 16 MiB at s = 4
    A = sscg.Matrix(ctx, S["rowptr"], S["col"], S["val"])
    opts = sscg.make_opts(s=4, tol=1e-8, maxit=100)
    need = C.c_size_t()
    assert ctx.lib.sscg_solve_workspace_bytes(A.h, C.byref(opts), C.byref(need)) == 0
    assert need.value > sscg.STATIC_SCRATCH_BYTES
    rc, x, _ = _static_solve(ctx, A, torch.from_numpy(S["b"]).cuda(), opts)
    assert rc == sscg.ERR_SPACE
    assert b"static scratch" in ctx.lib.sscg_last_error(ctx.h)
    assert np.all(x == 0.0)
