"""Spectral bounds of D^-1 A from a small network, trained on the device.

The Chebyshev basis and the Chebyshev polynomial preconditioner need an
interval [lambda_min, lambda_max] of D^-1 A (Section IV names the basis; the
paper does not say where the interval comes from).  `sscg_estimate_bounds`
gets it from Lanczos steps; this module trains a network that predicts it from
ten matrix features at the cost of one pass over the matrix.

Host logic only: the features, the forward and backward passes, the Adam
steps and the inference all run in libsscg's kernels (include/sscg.h, the
spectral-bound network section).  Training labels are extreme Ritz values
from many Lanczos steps on the device.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import inputs
from . import sscg

NFEAT = sscg.NFEAT
NOUT = 2


def _torch():
    return sscg._torch()


def _p(t):
    return C.c_void_p(t.data_ptr())


def xavier_init(d, h, o, seed):
    """theta with U(-a, a), a = sqrt(6/(fan_in+fan_out)), per weight matrix
    (Glorot and Bengio, 2010); biases zero.  Draws from splitmix64(seed)."""
    parts = []
    for k, (fi, fo) in enumerate(((d, h), (h, h), (h, o))):
        a = np.sqrt(6.0 / (fi + fo))
        parts.append(a * inputs.uniform(seed * 8 + k, fi * fo))
        parts.append(np.zeros(fo))
    return np.concatenate(parts)


class Network:
    """d -> h -> h -> o tanh network with FP64 parameters on the device."""

    def __init__(self, ctx: sscg.Context, d=NFEAT, h=64, o=NOUT, seed=0, theta=None):
        torch = _torch()
        self.ctx, self.d, self.h, self.o = ctx, d, h, o
        self.np = int(ctx.lib.sscg_mlp_nparams(d, h, o))
        th = xavier_init(d, h, o, seed) if theta is None else np.asarray(theta, dtype=np.float64)
        assert th.size == self.np
        self.theta = torch.from_numpy(th.copy()).cuda()
        self.x_mean = np.zeros(d)
        self.x_std = np.ones(d)
        self.y_mean = np.zeros(o)
        self.y_std = np.ones(o)

    def _ws(self, batch):
        torch = _torch()
        nb = C.c_size_t()
        self.ctx.check(self.ctx.lib.sscg_mlp_workspace_bytes(self.d, self.h, self.o, batch, C.byref(nb)))
        return torch.empty(nb.value, dtype=torch.uint8, device="cuda"), nb.value

    def forward(self, X):
        """Raw network outputs for raw (already normalised) inputs X (device, batch x d)."""
        torch = _torch()
        X = X.contiguous()
        B = X.shape[0]
        Y = torch.empty(B, self.o, dtype=torch.float64, device="cuda")
        ws, nb = self._ws(B)
        self.ctx.check(self.ctx.lib.sscg_mlp_forward(self.ctx.h, self.d, self.h, self.o, _p(self.theta), B, _p(X),
                                                     _p(Y), _p(ws), nb))
        return Y

    def loss_grad(self, X, T):
        torch = _torch()
        X, T = X.contiguous(), T.contiguous()
        B = X.shape[0]
        g = torch.empty(self.np, dtype=torch.float64, device="cuda")
        loss = C.c_double()
        ws, nb = self._ws(B)
        self.ctx.check(self.ctx.lib.sscg_mlp_loss_grad(self.ctx.h, self.d, self.h, self.o, _p(self.theta), B, _p(X),
                                                       _p(T), _p(g), C.byref(loss), _p(ws), nb))
        return loss.value, g

    def adam_step(self, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.ctx.check(self.ctx.lib.sscg_mlp_adam_step(self.ctx.h, self.np, _p(self.theta), _p(grad), _p(m), _p(v),
                                                       lr, b1, b2, eps, int(t)))

    def train(self, X, T, epochs, lr=3e-3, history=True):
        """Full-batch Adam on normalised inputs and targets (device tensors);
        returns the loss before each step (host array) when `history`."""
        torch = _torch()
        X, T = X.contiguous(), T.contiguous()
        B = X.shape[0]
        ws, nb = self._ws(B)
        hist = torch.empty(max(epochs, 1), dtype=torch.float64, device="cuda") if history else None
        self.ctx.check(self.ctx.lib.sscg_mlp_train(self.ctx.h, self.d, self.h, self.o, _p(self.theta), B, _p(X),
                                                   _p(T), int(epochs), float(lr),
                                                   _p(hist) if history else None, _p(ws), nb))
        return hist[:epochs].cpu().numpy() if history else None

    # -- the bounds model ------------------------------------------------

    def blob(self):
        """Device model blob [x_mean, x_std, y_mean, y_std, theta] for sscg_bounds_mlp."""
        torch = _torch()
        head = torch.from_numpy(np.concatenate([self.x_mean, self.x_std, self.y_mean, self.y_std])).cuda()
        return torch.cat([head, self.theta])

    def bounds(self, A: sscg.Matrix, blob=None):
        return A.bounds_mlp(self.h, self.blob() if blob is None else blob)

    def state(self):
        return dict(d=self.d, h=self.h, o=self.o, theta=self.theta.cpu().numpy(), x_mean=self.x_mean,
                    x_std=self.x_std, y_mean=self.y_mean, y_std=self.y_std)

    @classmethod
    def from_state(cls, ctx, st):
        net = cls(ctx, int(st["d"]), int(st["h"]), int(st["o"]), theta=st["theta"])
        for k in ("x_mean", "x_std", "y_mean", "y_std"):
            setattr(net, k, np.asarray(st[k], dtype=np.float64))
        return net


@dataclass
class Sample:
    kind: str
    N: int
    sigma: float
    ell: float
    seed: int


def default_samples(sizes=(8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128), seeds_per=3, seed0=100):
    """Training recipe: constant 7- and 27-point stencils at every size, and
    variable-coefficient 7-point fields with sigma in {0.5, 1, 1.5, 2} and
    smoothing length in {2, 4, 8}, `seeds_per` draws per size."""
    out = []
    rng = seed0
    for N in sizes:
        out.append(Sample("poisson7", N, 0.0, 4.0, 0))
        out.append(Sample("poisson27", N, 0.0, 4.0, 0))
        for r in range(seeds_per):
            sig = (0.5, 1.0, 1.5, 2.0)[(r + N) % 4]
            ell = (2.0, 4.0, 8.0)[(r + 2 * N) % 3]
            out.append(Sample("varcoef7", N, sig, ell, rng))
            rng += 1
    return out


def matrix_for(ctx, smp: Sample):
    if smp.kind == "varcoef7":
        rowptr, col, val = inputs.varcoef7(smp.N, smp.sigma, smp.seed, smp.ell)
    elif smp.kind == "poisson7":
        rowptr, col, val = inputs.poisson7(smp.N)
    elif smp.kind == "poisson27":
        rowptr, col, val = inputs.poisson27(smp.N)
    else:
        raise ValueError(smp.kind)
    return sscg.Matrix(ctx, rowptr, col, val)


def label_steps(n, steps=None):
    """Lanczos steps for a label: about 8 per grid line plus 100 (the smallest
    eigenvalue of a grid operator converges after O(N) steps), at most n/2."""
    if steps is None:
        steps = 8 * round(n ** (1.0 / 3.0)) + 100
    return int(min(steps, max(8, n // 2)))


def ritz_label(A: sscg.Matrix, steps=None, seed=1):
    """(ln lambda_min, ln lambda_max) of D^-1 A from Lanczos on the device."""
    A.set_preconditioner("jacobi")
    r0 = A.ctx.uniform(A.n, seed)
    lo, hi = A.estimate_bounds(label_steps(A.n, steps), r0=r0)
    return np.log(lo), np.log(hi)


def dataset(ctx, samples, steps=None):
    """Features (host, len x NFEAT) and labels (host, len x 2) of `samples`."""
    X = np.zeros((len(samples), NFEAT))
    T = np.zeros((len(samples), NOUT))
    for i, smp in enumerate(samples):
        A = matrix_for(ctx, smp)
        X[i] = A.features()
        T[i] = ritz_label(A, steps)
        A.close()
    return X, T


def fit(ctx, X, T, hidden=64, epochs=4000, lr=3e-3, seed=0):
    """Normalise, train on the device, return (network, loss history)."""
    torch = _torch()
    net = Network(ctx, X.shape[1], hidden, T.shape[1], seed=seed)
    net.x_mean = X.mean(axis=0)
    net.x_std = np.where(X.std(axis=0) > 1e-12, X.std(axis=0), 1.0)
    net.y_mean = T.mean(axis=0)
    net.y_std = np.where(T.std(axis=0) > 1e-12, T.std(axis=0), 1.0)
    Xn = torch.from_numpy((X - net.x_mean) / net.x_std).cuda()
    Tn = torch.from_numpy((T - net.y_mean) / net.y_std).cuda()
    hist = net.train(Xn, Tn, epochs, lr)
    return net, hist
