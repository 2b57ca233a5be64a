"""The measurement probes of include/sscg_probe.h: the throughput probe
reports a positive rate, and the small-solve latency probe runs the
library's s x s routines to completion (no failed factorisation) with
positive cycle counts, and rejects out-of-range arguments."""
import pytest

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


def test_throughput_probe_reports_a_rate(ctx):
    ops, ms = ctx.probe_rate("dfma", 1000)
    assert ops > 0 and ms > 0


@pytest.mark.parametrize("s", [1, 2, 4, 8])
def test_small_solve_probe_runs_the_solves(ctx, s):
    c = ctx.probe_small_solve(s, 20)
    assert set(c) == {"cholesky", "solve_1", "solve_s", "monomial_step0"}
    assert all(v > 0 for v in c.values()), c
    # the first-step form factors the moment matrix and solves once
    assert c["monomial_step0"] > c["solve_1"]


@pytest.mark.parametrize("s,reps", [(0, 10), (9, 10), (4, 0), (4, 100001)])
def test_small_solve_probe_rejects_bad_arguments(ctx, s, reps):
    with pytest.raises(sscg.SscgError):
        ctx.probe_small_solve(s, reps)
