"""The spectral-bound network on the device: features, forward, gradient,
Adam and inference against the FP64 oracle, training quality, and the gain
over Lanczos bounds for the Chebyshev basis and preconditioner at 128^3."""
import time

import numpy as np
import pytest

import oracle
from paper_2501_03743_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2501_03743_gb300 import spectral, sscg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_2501_03743_gb300 import build

    build.build()
    return sscg.Context()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def csr_of(S):
    return S["rowptr"], S["col"], S["val"]


# ---------------------------------------------------------------- features

FEATURE_CASES = [
    ("poisson7", 9, 0.0, 4.0, 0),
    ("poisson27", 7, 0.0, 4.0, 0),
    ("varcoef7", 20, 1.5, 4.0, 3),
    ("varcoef7", 33, 2.0, 2.0, 4),   # 35,937 rows: many CTAs and a ragged tail
    ("varcoef7", 64, 1.0, 8.0, 5),
]


@pytest.mark.parametrize("case", FEATURE_CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def test_features_match_oracle(ctx, case):
    kind, N, sigma, ell, seed = case
    smp = spectral.Sample(kind, N, sigma, ell, seed)
    A = spectral.matrix_for(ctx, smp)
    got = A.features()
    if kind == "varcoef7":
        csr = inputs.varcoef7(N, sigma, seed, ell)
    else:
        csr = getattr(inputs, kind)(N)
    want = oracle.features(oracle.Matrix(*csr))
    # logarithms in FP32 on the device: about 1e-7 relative per value
    assert np.all(np.abs(got - want) <= 2e-6 * (1 + np.abs(want))), (got, want)


def test_features_dense_random_and_diagonal(ctx):
    rng = inputs.uniform(21, 60 * 60).reshape(60, 60)
    S = np.where(np.abs(rng) < 0.2, rng, 0.0)
    S = np.triu(S, 1)
    S = S + S.T
    D = S + np.diag(np.abs(S).sum(1) + 0.3 + np.abs(inputs.uniform(22, 60)))
    M = oracle.Matrix.from_dense(D)
    A = sscg.Matrix(ctx, M.rowptr, M.col, M.val)
    want = oracle.features(M)
    assert np.all(np.abs(A.features() - want) <= 2e-6 * (1 + np.abs(want)))
    # no off-diagonal entries: f6..f9 are zero
    d = np.exp(inputs.uniform(23, 17))
    M = oracle.Matrix.from_dense(np.diag(d))
    A = sscg.Matrix(ctx, M.rowptr, M.col, M.val)
    got = A.features()
    want = oracle.features(M)
    assert np.all(np.abs(got - want) <= 2e-6 * (1 + np.abs(want)))
    assert np.all(got[6:] == 0.0)


# ------------------------------------------------------- network parity

SHAPES = [(10, 64, 2, 100), (10, 64, 2, 1), (3, 1, 1, 5), (7, 33, 3, 257)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_forward_and_gradient_match_oracle(ctx, shape):
    d, h, o, B = shape
    npar = oracle.mlp_nparams(d, h, o)
    theta = 0.5 * inputs.uniform(31 + d, npar)
    X = inputs.uniform(32 + h, B * d).reshape(B, d)
    T = inputs.uniform(33 + o, B * o).reshape(B, o)
    net = spectral.Network(ctx, d, h, o, theta=theta)
    Y = net.forward(dev(X)).cpu().numpy()
    assert rel(Y, oracle.mlp_forward(d, h, o, theta, X)) < 1e-13
    loss, g = net.loss_grad(dev(X), dev(T))
    loss_o, g_o = oracle.mlp_loss_grad(d, h, o, theta, X, T)
    assert abs(loss - loss_o) <= 1e-13 * abs(loss_o)
    assert rel(g.cpu().numpy(), g_o) < 1e-12


def test_adam_steps_match_oracle(ctx):
    npar = 1000
    theta = inputs.uniform(41, npar)
    net_t = dev(theta)
    m_t, v_t = torch.zeros(npar, dtype=torch.float64, device="cuda"), torch.zeros(npar, dtype=torch.float64,
                                                                                   device="cuda")
    m, v = np.zeros(npar), np.zeros(npar)
    th = theta.copy()
    net = spectral.Network(ctx, 10, 8, 2)  # only its context binding is used
    for t in range(1, 6):
        g = inputs.uniform(42 + t, npar) * (10.0 ** (t - 3))
        net.ctx.check(net.ctx.lib.sscg_mlp_adam_step(net.ctx.h, npar, spectral._p(net_t), spectral._p(dev(g)),
                                                     spectral._p(m_t), spectral._p(v_t), 0.01, 0.9, 0.999, 1e-8, t))
        oracle.adam_step(th, g, m, v, t, lr=0.01)
    assert rel(net_t.cpu().numpy(), th) < 1e-14
    assert rel(m_t.cpu().numpy(), m) < 1e-14 and rel(v_t.cpu().numpy(), v) < 1e-14


def test_training_loop_matches_oracle(ctx):
    """sscg_mlp_train = the oracle's gradient + Adam, step for step."""
    d, h, o, B, epochs, lr = 10, 16, 2, 40, 25, 5e-3
    theta0 = spectral.xavier_init(d, h, o, seed=3)
    X = inputs.uniform(51, B * d).reshape(B, d)
    T = inputs.uniform(52, B * o).reshape(B, o)
    net = spectral.Network(ctx, d, h, o, theta=theta0)
    hist = net.train(dev(X), dev(T), epochs, lr)
    th, m, v = theta0.copy(), np.zeros_like(theta0), np.zeros_like(theta0)
    losses = []
    for t in range(1, epochs + 1):
        loss, g = oracle.mlp_loss_grad(d, h, o, th, X, T)
        losses.append(loss)
        oracle.adam_step(th, g, m, v, t, lr=lr)
    assert rel(hist, losses) < 1e-11
    assert rel(net.theta.cpu().numpy(), th) < 1e-10


def test_inference_kernel_matches_oracle(ctx):
    """sscg_bounds_mlp = exp(de-normalised network(normalised features))."""
    net = spectral.Network(ctx, sscg.NFEAT, 48, 2, seed=9)
    net.theta = dev(0.3 * inputs.uniform(61, net.np))
    net.x_mean = inputs.uniform(62, sscg.NFEAT)
    net.x_std = 1.5 + inputs.uniform(63, sscg.NFEAT)
    net.y_mean = np.array([-6.0, 0.6])  # keeps lambda_min well below lambda_max
    net.y_std = np.array([1.2, 0.1])
    A = spectral.matrix_for(ctx, spectral.Sample("varcoef7", 24, 1.0, 4.0, 7))
    lo, hi = net.bounds(A)
    f = oracle.features(oracle.Matrix(*inputs.varcoef7(24, 1.0, 7, 4.0)))
    y = oracle.mlp_forward(sscg.NFEAT, 48, 2, net.theta.cpu().numpy(), ((f - net.x_mean) / net.x_std)[None, :])[0]
    want = np.exp(y * net.y_std + net.y_mean)
    assert abs(lo / want[0] - 1) < 1e-5 and abs(hi / want[1] - 1) < 1e-5


def test_bounds_mlp_rejects_bad_arguments(ctx):
    A = spectral.matrix_for(ctx, spectral.Sample("poisson7", 6, 0.0, 4.0, 0))
    blob = torch.zeros(4 * sscg.NFEAT + 4 + 5000, dtype=torch.float64, device="cuda")
    with pytest.raises(sscg.SscgError):
        A.bounds_mlp(0, blob)
    with pytest.raises(sscg.SscgError):
        A.bounds_mlp(300, blob)
    # an all-zero model predicts lambda_min = lambda_max = 1: an empty interval
    with pytest.raises(sscg.SscgError) as e:
        A.bounds_mlp(16, blob)
    assert "interval" in str(e.value)


# ------------------------------------------------------ training quality

@pytest.fixture(scope="module")
def trained(ctx):
    samples = spectral.default_samples(seeds_per=6)
    X, T = spectral.dataset(ctx, samples)
    net, hist = spectral.fit(ctx, X, T, hidden=64, epochs=4000, lr=3e-3, seed=0)
    return dict(samples=samples, X=X, T=T, net=net, hist=hist)


def test_labels_match_closed_forms(trained):
    """The Lanczos labels of the constant stencils reach the exact spectrum of
    D^-1 A (approached from inside)."""
    for smp, t in zip(trained["samples"], trained["T"]):
        if smp.kind == "varcoef7":
            continue
        lo, hi = inputs.closed_form_bounds(smp.kind, smp.N)
        diag = 6.0 if smp.kind == "poisson7" else 26.0
        lo, hi = lo / diag, hi / diag
        assert np.log(lo) - 1e-9 <= t[0] <= np.log(lo) + 0.02, (smp, np.exp(t[0]), lo)
        assert np.log(hi) - 0.01 <= t[1] <= np.log(hi) + 1e-9, (smp, np.exp(t[1]), hi)


def test_training_converges(trained):
    hist = trained["hist"]
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 1e-3 * hist[0]


HELD_OUT = [(24, 1.0, 4.0), (40, 1.5, 2.0), (64, 0.5, 8.0), (96, 2.0, 4.0), (56, 1.0, 4.0), (72, 2.0, 8.0)]


def test_network_bounds_on_held_out_fields(ctx, trained):
    """Unseen variable-coefficient fields (new seeds) at sizes inside the
    training range.  lambda_max is predicted to 2%; lambda_min, which depends
    on where the field's low-conductivity regions sit, to within a factor of
    6.  The Chebyshev basis does not need more: with the network's interval
    the s = 12 solve takes the same number of steps as with the exact one."""
    net = trained["net"]
    blob = net.blob()
    for i, (N, sig, ell) in enumerate(HELD_OUT):
        smp = spectral.Sample("varcoef7", N, sig, ell, 9000 + i)
        A = spectral.matrix_for(ctx, smp)
        lo, hi = net.bounds(A, blob)
        tl, th = spectral.ritz_label(A)
        assert abs(np.log(hi) - th) < 0.02, (smp, hi, np.exp(th))
        assert abs(np.log(lo) - tl) < np.log(6.0), (smp, lo, np.exp(tl))
        S = inputs.varcoef7(N, sig, 9000 + i, ell)
        b = dev(inputs.matvec(*S, inputs.uniform(5, A.n)))
        steps = []
        for bnd in ((0.95 * lo, 1.05 * hi), (0.95 * np.exp(tl), 1.05 * np.exp(th))):
            x = torch.zeros_like(b)
            r = sscg.Solver(A, s=12, basis="chebyshev", basis_bounds=bnd, tol=1e-8, maxit=2000).solve(b, x)
            assert r.converged and r.rel_res_true < 1e-7
            steps.append(r.outer_iters)
        assert abs(steps[0] - steps[1]) <= 1, (smp, steps)


def test_gain_over_lanczos_at_128(ctx, trained):
    """At 128^3 (variable coefficients, an unseen field) the network's bounds
    cost one pass over the matrix instead of 20 Lanczos steps, and a
    Chebyshev-basis solve at s = 12 that takes its interval from the network
    (attached to the matrix) converges in the same number of steps as one that
    estimates it by Lanczos, where the monomial basis breaks down."""
    net = trained["net"]
    blob = net.blob()
    smp = spectral.Sample("varcoef7", 128, 1.0, 4.0, 9999)
    A = spectral.matrix_for(ctx, smp)
    S = inputs.varcoef7(128, 1.0, 9999, 4.0)
    b = dev(inputs.matvec(*S, inputs.uniform(77, A.n)))

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) / reps

    _, t_lanczos = timed(lambda: A.estimate_bounds(20))
    _, t_mlp = timed(lambda: net.bounds(A, blob))
    assert t_mlp < t_lanczos / 3, (t_mlp, t_lanczos)

    def solve(**kw):
        x = torch.zeros_like(b)
        return sscg.Solver(A, tol=1e-8, maxit=2000, **kw).solve(b, x)

    r_lanczos = solve(s=12, basis="chebyshev")
    A.set_bounds_model(net.h, blob)
    r_net = solve(s=12, basis="chebyshev")
    A.set_bounds_model(net.h, None)
    r_pcg = sscg.Solver(A, method="pcg", tol=1e-8, maxit=20000).solve(b, torch.zeros_like(b))
    assert r_lanczos.converged and r_net.converged
    assert r_net.rel_res_true < 1e-7
    assert abs(r_net.outer_iters - r_lanczos.outer_iters) <= 1
    assert r_net.equiv_iters <= r_pcg.equiv_iters + 24
    assert solve(s=12).status == sscg.BREAKDOWN


def test_attached_model_needs_jacobi_and_valid_width(ctx, trained):
    net = trained["net"]
    A = spectral.matrix_for(ctx, spectral.Sample("poisson7", 12, 0.0, 4.0, 0))
    with pytest.raises(sscg.SscgError):
        A.set_bounds_model(0, net.blob())
    A.set_bounds_model(net.h, net.blob())
    b = dev(inputs.matvec(*inputs.poisson7(12), inputs.uniform(3, A.n)))
    r = sscg.Solver(A, s=8, basis="chebyshev", tol=1e-9, maxit=500).solve(b, torch.zeros_like(b))
    assert r.converged and r.rel_res_true < 1e-8
    # under a Chebyshev preconditioner the solve estimates by Lanczos instead
    lo, hi = inputs.closed_form_bounds("poisson7", 12)
    A.set_preconditioner("cheb", 3, 0.9 * lo / 6, 1.05 * hi / 6)
    r = sscg.Solver(A, s=4, basis="chebyshev", tol=1e-9, maxit=500).solve(b, torch.zeros_like(b))
    assert r.converged and r.rel_res_true < 1e-8
