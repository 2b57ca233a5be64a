"""The seeded input generators: the torch stencil builder reproduces the
numpy one exactly, and the serving mix is deterministic and in range."""
import numpy as np
import pytest

from paper_2501_03743_gb300 import inputs


@pytest.mark.parametrize("kind", ["poisson7", "poisson27"])
@pytest.mark.parametrize("N", [1, 2, 5, 11])
def test_torch_stencil_matches_numpy(kind, N):
    pytest.importorskip("torch")
    ref = getattr(inputs, kind)(N)
    got = [t.numpy() for t in inputs.stencil_torch(kind, N, "cpu")]
    for a, b in zip(ref, got):
        assert a.dtype == b.dtype and np.array_equal(a, b)


def test_batch_spec_is_seeded_and_in_range():
    a = inputs.batch_spec(64, seed=7)
    assert a == inputs.batch_spec(64, seed=7)
    assert a != inputs.batch_spec(64, seed=8)
    assert len(a) == 64
    for e in a:
        assert 32 <= e["N"] <= 160 and 1 <= e["nrhs"] <= 8
        assert e["kind"] in ("poisson7", "poisson27", "varcoef7") and e["sigma"] in (0.5, 1.0, 2.0, 3.0)
    assert {e["kind"] for e in a} == {"poisson7", "poisson27", "varcoef7"}
    r = inputs.batch_csr(dict(kind="varcoef7", N=6, sigma=2.0, field_seed=3, nrhs=1))
    ref = inputs.varcoef7(6, 2.0, 3)
    assert all(np.array_equal(x, y) for x, y in zip(r, ref))


def test_aniso7_couplings():
    """The anisotropic stencil: symmetric, centre 14, couplings -1/-2/-4 along
    x/y/z (strides 1, N, N^2), positive definite."""
    import scipy.sparse as sp

    N = 5
    rowptr, col, val = inputs.aniso7(N)
    A = sp.csr_matrix((val, col, rowptr), shape=(N ** 3, N ** 3)).toarray()
    assert np.array_equal(A, A.T)
    i = 2 + 2 * N + 2 * N * N  # an interior node
    assert A[i, i] == 14.0
    assert A[i, i - 1] == A[i, i + 1] == -1.0
    assert A[i, i - N] == A[i, i + N] == -2.0
    assert A[i, i - N * N] == A[i, i + N * N] == -4.0
    assert np.count_nonzero(A[i]) == 7
    assert np.linalg.eigvalsh(A).min() > 0.0


def test_aniso7_closed_form_spectrum():
    """The anisotropic stencil is a Kronecker sum of three 1-D Dirichlet
    operators: eigenvalues 14 - 2 cos(a) - 4 cos(b) - 8 cos(c) over the sine
    modes a, b, c = pi k / (N + 1)."""
    import scipy.sparse as sp

    N = 4
    rowptr, col, val = inputs.aniso7(N)
    A = sp.csr_matrix((val, col, rowptr), shape=(N ** 3, N ** 3)).toarray()
    th = np.pi * np.arange(1, N + 1) / (N + 1)
    c = np.cos(th)
    lam = 14.0 - 2.0 * c[:, None, None] - 4.0 * c[None, :, None] - 8.0 * c[None, None, :]
    assert np.allclose(np.sort(lam.ravel()), np.linalg.eigvalsh(A), atol=1e-12)
