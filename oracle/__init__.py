"""Python access to the FP64 CPU oracle (``sscg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing in the CUDA
library imports this package, and this package imports nothing from it.

The shared library is compiled on first use (``build()``) with plain gcc,
``-O2 -ffp-contract=off`` (identical rounding on x86 and Arm hosts) and
OpenMP when the compiler offers it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sscg_oracle.c")
_HDR = os.path.join(_HERE, "sscg_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

PREC = {"none": 0, "jacobi": 1, "cheb": 2}
BASIS = {"monomial": 0, "chebyshev": 1, "newton": 2}
OK, NOT_CONVERGED, BREAKDOWN, ERR_INVALID = 0, 1, 2, -1


def build(force: bool = False) -> str:
    """Compile the oracle if its object is missing or older than its sources."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = force or not os.path.exists(_OUT) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_OUT)
    if stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, _OUT)
    return _OUT


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class _Prec(C.Structure):
    _fields_ = [("kind", C.c_int), ("degree", C.c_int), ("lmin", C.c_double), ("lmax", C.c_double)]


class _Res(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("relres", C.c_double),
                ("hist", C.c_void_p), ("hist_cap", C.c_int), ("hist_len", C.c_int)]


class _Trace(C.Structure):
    _fields_ = [("cap", C.c_int)] + [(k, C.c_void_p) for k in
                ("U", "AU", "P", "AP", "r", "x", "W", "alpha", "beta", "b1", "vm")] + [("len", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        # SSCG_ORACLE_LIB points the tests at an alternative build of the same
        # source (the mutation test plants one mistake per build).
        L = C.CDLL(os.environ.get("SSCG_ORACLE_LIB") or build())
        vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
        P = C.POINTER
        L.orc_spmv.argtypes = [P(_Csr), vp, vp]
        L.orc_dot.argtypes = [i64, vp, vp]; L.orc_dot.restype = dbl
        L.orc_diag.argtypes = [P(_Csr), vp]
        L.orc_prec_apply.argtypes = [P(_Csr), P(_Prec), vp, vp]
        L.orc_pcg.argtypes = [P(_Csr), P(_Prec), vp, vp, dbl, i32, P(_Res), vp, vp]
        L.orc_pcgs.argtypes = [P(_Csr), P(_Prec), vp, vp, i32, dbl, i32, P(_Res), P(_Trace)]
        L.orc_pcgs_gram.argtypes = [P(_Csr), P(_Prec), vp, vp, i32, i32, dbl, dbl, dbl, i32, P(_Res), P(_Trace)]
        L.orc_pfcg.argtypes = [P(_Csr), P(_Prec), vp, vp, dbl, i32, P(_Res)]
        L.orc_newton_shifts.argtypes = [i32, dbl, dbl, vp, P(dbl)]
        L.orc_chol_solve.argtypes = [i32, vp, i32, vp, vp]
        L.orc_tridiag_eig_extremes.argtypes = [i32, vp, vp, P(dbl), P(dbl)]
        L.orc_lanczos_bounds.argtypes = [P(_Csr), P(_Prec), vp, i32, P(dbl), P(dbl)]
        L.orc_mlp_nparams.argtypes = [i32, i32, i32]; L.orc_mlp_nparams.restype = i64
        L.orc_mlp_forward.argtypes = [i32, i32, i32, vp, i32, vp, vp]
        L.orc_mlp_loss_grad.argtypes = [i32, i32, i32, vp, i32, vp, vp, vp]; L.orc_mlp_loss_grad.restype = dbl
        L.orc_features.argtypes = [P(_Csr), vp]; L.orc_features.restype = i32
        L.orc_adam_step.argtypes = [i64, vp, vp, vp, vp, dbl, dbl, dbl, dbl, i32]
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Matrix:
    """CSR matrix view kept alive for the oracle (int32 indices, FP64 values)."""

    def __init__(self, rowptr, col, val):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = _f64(val)
        self.n = len(self.rowptr) - 1
        self.c = _Csr(self.n, _ptr(self.rowptr).value, _ptr(self.col).value, _ptr(self.val).value)

    @classmethod
    def from_dense(cls, D):
        D = np.asarray(D, dtype=np.float64)
        rows, cols = np.nonzero(D)
        rowptr = np.zeros(D.shape[0] + 1, dtype=np.int64)
        np.add.at(rowptr, rows + 1, 1)
        return cls(np.cumsum(rowptr), cols, D[rows, cols])

    def to_dense(self):
        D = np.zeros((self.n, self.n))
        for i in range(self.n):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                D[i, self.col[k]] += self.val[k]
        return D


def as_matrix(A) -> Matrix:
    if isinstance(A, Matrix):
        return A
    if isinstance(A, dict):
        return Matrix(A["rowptr"], A["col"], A["val"])
    return Matrix(*A)


def _prec(prec) -> _Prec:
    if prec is None:
        return _Prec(0, 0, 0.0, 0.0)
    if isinstance(prec, str):
        return _Prec(PREC[prec], 0, 0.0, 0.0)
    return _Prec(PREC[prec["kind"]], int(prec.get("degree", 0)), float(prec.get("lmin", 0.0)), float(prec.get("lmax", 0.0)))


@dataclass
class Result:
    x: np.ndarray
    status: int
    iters: int
    relres: float
    hist: np.ndarray
    extra: dict = field(default_factory=dict)


def _res(cap):
    h = np.zeros(cap + 2)
    return h, _Res(0, 0, 0.0, _ptr(h).value, cap + 2, 0)


def spmv(A, x):
    A = as_matrix(A); x = _f64(x); y = np.empty(A.n)
    lib().orc_spmv(C.byref(A.c), _ptr(x), _ptr(y))
    return y


def diag(A):
    A = as_matrix(A); d = np.empty(A.n)
    lib().orc_diag(C.byref(A.c), _ptr(d))
    return d


def prec_apply(A, prec, r):
    A = as_matrix(A); r = _f64(r); z = np.empty(A.n); p = _prec(prec)
    st = lib().orc_prec_apply(C.byref(A.c), C.byref(p), _ptr(r), _ptr(z))
    if st != OK:
        raise ValueError("invalid preconditioner")
    return z


def pcg(A, b, x0=None, prec="jacobi", tol=1e-8, maxit=10000, coeffs=False) -> Result:
    """Algorithm 1."""
    A = as_matrix(A); b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    h, res = _res(maxit)
    p = _prec(prec)
    ca = np.zeros(max(maxit, 1)); cb = np.zeros(max(maxit, 1))
    lib().orc_pcg(C.byref(A.c), C.byref(p), _ptr(b), _ptr(x), tol, maxit, C.byref(res),
                  _ptr(ca) if coeffs else None, _ptr(cb) if coeffs else None)
    out = Result(x, res.status, res.iters, res.relres, h[:res.hist_len].copy())
    if coeffs:
        out.extra = dict(alpha=ca[:res.iters].copy(), beta=cb[:res.iters].copy())
    return out


def pfcg(A, b, x0=None, prec="jacobi", tol=1e-8, maxit=10000) -> Result:
    """Algorithm 2."""
    A = as_matrix(A); b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    h, res = _res(maxit)
    p = _prec(prec)
    lib().orc_pfcg(C.byref(A.c), C.byref(p), _ptr(b), _ptr(x), tol, maxit, C.byref(res))
    return Result(x, res.status, res.iters, res.relres, h[:res.hist_len].copy())


def _trace(n, s, cap):
    if not cap:
        return None, None
    bufs = dict(U=np.zeros((cap, s, n)), AU=np.zeros((cap, s, n)), P=np.zeros((cap, s, n)), AP=np.zeros((cap, s, n)),
                r=np.zeros((cap, n)), x=np.zeros((cap, n)), W=np.zeros((cap, s, s)), alpha=np.zeros((cap, s)),
                beta=np.zeros((cap, s, s)), b1=np.zeros((cap, s, s)), vm=np.zeros((cap, 2 * s)))
    t = _Trace(cap, *[_ptr(bufs[k]).value for k in ("U", "AU", "P", "AP", "r", "x", "W", "alpha", "beta", "b1", "vm")], 0)
    return t, bufs


def _untrace(t, bufs):
    """Blocks come back as [step][column][row]; transpose to n x s per step,
    and W/beta/b1 (column-major in C) to row-major."""
    if t is None:
        return {}
    L = t.len
    out = {k: v[:L].copy() for k, v in bufs.items()}
    for k in ("U", "AU", "P", "AP"):
        out[k] = np.transpose(out[k], (0, 2, 1))
    for k in ("W", "beta", "b1"):
        out[k] = np.transpose(out[k], (0, 2, 1))
    return out


def pcgs(A, b, s, x0=None, prec="jacobi", tol=1e-8, maxit=10000, trace=0) -> Result:
    """Algorithm 3 with Algorithms 4-6 (monomial basis)."""
    A = as_matrix(A); b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    h, res = _res(maxit)
    p = _prec(prec)
    t, bufs = _trace(A.n, s, trace)
    lib().orc_pcgs(C.byref(A.c), C.byref(p), _ptr(b), _ptr(x), s, tol, maxit, C.byref(res),
                   C.byref(t) if t is not None else None)
    return Result(x, res.status, res.iters, res.relres, h[:res.hist_len].copy(), _untrace(t, bufs))


def pcgs_gram(A, b, s, basis="monomial", bounds=(0.0, 0.0), x0=None, prec="jacobi", tol=1e-8,
              maxit=10000, trace=0) -> Result:
    """The s-step method with directly formed Gram blocks, any basis."""
    A = as_matrix(A); b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    h, res = _res(maxit)
    p = _prec(prec)
    t, bufs = _trace(A.n, s, trace)
    lib().orc_pcgs_gram(C.byref(A.c), C.byref(p), _ptr(b), _ptr(x), s, BASIS[basis], float(bounds[0]),
                        float(bounds[1]), tol, maxit, C.byref(res), C.byref(t) if t is not None else None)
    return Result(x, res.status, res.iters, res.relres, h[:res.hist_len].copy(), _untrace(t, bufs))


def newton_shifts(s, lo, hi):
    """(theta[0..s-2], sigma) of the Newton basis over [lo, hi] (orc_newton_shifts)."""
    theta = np.zeros(max(s - 1, 1))
    sig = C.c_double()
    st = lib().orc_newton_shifts(int(s), float(lo), float(hi), _ptr(theta), C.byref(sig))
    if st != OK:
        raise ValueError("bad Newton-shift arguments")
    return theta[: s - 1].copy(), sig.value


def chol_solve(Adense, B):
    A = np.asfortranarray(Adense, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    vecin = B.ndim == 1
    Bf = np.asfortranarray(B.reshape(len(B), -1))
    X = np.zeros_like(Bf, order="F")
    st = lib().orc_chol_solve(A.shape[0], _ptr(A), Bf.shape[1], _ptr(Bf), _ptr(X))
    return st, (X[:, 0] if vecin else X)


def tridiag_extremes(d, e):
    d = _f64(d); e = _f64(np.append(e, 0.0))
    lo, hi = C.c_double(), C.c_double()
    lib().orc_tridiag_eig_extremes(len(d), _ptr(d), _ptr(e), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def lanczos_bounds(A, r0, k, prec="jacobi"):
    A = as_matrix(A); r0 = _f64(r0)
    lo, hi = C.c_double(), C.c_double()
    p = _prec(prec)
    st = lib().orc_lanczos_bounds(C.byref(A.c), C.byref(p), _ptr(r0), k, C.byref(lo), C.byref(hi))
    if st != OK:
        raise RuntimeError(f"lanczos failed: {st}")
    return lo.value, hi.value


def mlp_nparams(d, h, o):
    return int(lib().orc_mlp_nparams(d, h, o))


def mlp_forward(d, h, o, theta, X):
    theta = _f64(theta); X = _f64(X).reshape(-1, d); Y = np.zeros((X.shape[0], o))
    lib().orc_mlp_forward(d, h, o, _ptr(theta), X.shape[0], _ptr(X), _ptr(Y))
    return Y


def mlp_loss_grad(d, h, o, theta, X, T):
    theta = _f64(theta); X = _f64(X).reshape(-1, d); T = _f64(T).reshape(-1, o)
    g = np.zeros(mlp_nparams(d, h, o))
    loss = lib().orc_mlp_loss_grad(d, h, o, _ptr(theta), X.shape[0], _ptr(X), _ptr(T), _ptr(g))
    return loss, g


def num_threads() -> int:
    return int(lib().orc_num_threads())


NFEAT = 10


def features(A):
    """The ten matrix features of the spectral-bound network (orc_features)."""
    A = as_matrix(A)
    f = np.zeros(NFEAT)
    if lib().orc_features(C.byref(A.c), _ptr(f)) != 0:
        raise ValueError("non-positive diagonal")
    return f


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on theta, m, v (orc_adam_step)."""
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib().orc_adam_step(theta.size, _ptr(theta), _ptr(g), _ptr(m), _ptr(v), lr, b1, b2, eps, int(t))
