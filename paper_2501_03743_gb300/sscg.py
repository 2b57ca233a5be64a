"""Python binding of libsscg (include/sscg.h): argument marshalling only.

PyTorch supplies device memory (matrix storage, solve workspace, vectors)
and the CUDA stream; every numerical step runs in the library's kernels.
There is no CPU fallback: importing this module on a machine without the
built library, or calling a solve without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsscg.so")

OK, NOT_CONVERGED, BREAKDOWN, TIMEOUT = 0, 1, 2, 3
ERR_INVALID, ERR_NOT_SPD, ERR_CUDA, ERR_SPACE, ERR_NONFINITE = -1, -2, -3, -4, -5
BASIS = {"monomial": 0, "chebyshev": 1, "newton": 2}
PREC = {"none": 0, "jacobi": 1, "cheb": 2}
ARITH = {"f64": 0, "df64": 1, "mixed": 2}
HOST_VECTORS = 0x1
HOST_ARRAYS = 0x1
MAT_CSR_ONLY = 0x2
FORMAT = {0: "csr", 1: "dia_const"}

# Every symbol include/sscg.h declares, for the export check.
EXPORTS = (
    "sscg_create", "sscg_destroy", "sscg_last_error", "sscg_status_str", "sscg_version",
    "sscg_mat_storage_bytes", "sscg_mat_create_csr", "sscg_mat_destroy", "sscg_mat_props_get",
    "sscg_set_preconditioner", "sscg_solve_workspace_bytes", "sscg_solve", "sscg_pcg_workspace_bytes",
    "sscg_pcg_solve", "sscg_spmv", "sscg_bounds_workspace_bytes", "sscg_estimate_bounds", "sscg_uniform",
    "sscg_solve_static", "sscg_features_workspace_bytes", "sscg_mat_features", "sscg_mlp_nparams",
    "sscg_mlp_workspace_bytes", "sscg_mlp_forward", "sscg_mlp_loss_grad", "sscg_mlp_adam_step", "sscg_mlp_train",
    "sscg_bounds_mlp", "sscg_set_bounds_model", "sscg_batch_workspace_bytes", "sscg_batch_create",
    "sscg_batch_destroy", "sscg_batch_solve", "sscg_batch_props", "sscg_batch_launches",
    "sscg_probe_rate", "sscg_batch_inject_barrier_fault", "sscg_pfcg_workspace_bytes", "sscg_pfcg_solve",
    "sscg_newton_shifts", "sscg_probe_small_solve",
)
# Probe kinds of include/sscg_probe.h.
PROBE = {"dfma": 0, "dadd": 1, "dmul": 2, "dmma": 3, "dfma_dmma": 4, "ffma": 5, "ialu": 6, "imad": 7, "imad_wide": 8, "i2f64": 9,
         "f2i64": 10}
BATCH_MAX_RHS = 8
BATCH_PERSISTENT = 0x10
BATCH_MAX_S = 8
NFEAT = 10
STATIC_SCRATCH_BYTES = 16 << 20


class SscgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sscg error {code}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("s", C.c_int), ("basis", C.c_int), ("basis_lmin", C.c_double), ("basis_lmax", C.c_double),
                ("tol", C.c_double), ("maxit", C.c_int), ("arith", C.c_int), ("replace_every", C.c_int),
                ("flags", C.c_uint)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("equiv_iters", C.c_int64),
                ("rel_res_recursive", C.c_double), ("rel_res_true", C.c_double), ("hist", C.c_void_p),
                ("hist_cap", C.c_int), ("hist_len", C.c_int), ("kernel_launches", C.c_int64),
                ("t_init_ms", C.c_double), ("t_mpk_ms", C.c_double), ("t_update_ms", C.c_double),
                ("t_dir_ms", C.c_double), ("t_final_ms", C.c_double), ("n_mpk", C.c_int64),
                ("n_update", C.c_int64), ("n_dir", C.c_int64), ("s_final", C.c_int)]


PROFILE = 0x2
_PROFILE_FIELDS = ("kernel_launches", "t_init_ms", "t_mpk_ms", "t_update_ms", "t_dir_ms", "t_final_ms", "n_mpk",
                   "n_update", "n_dir", "s_final")


class MatProps(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("bandwidth", C.c_int64), ("values_exact_fp32", C.c_int),
                ("max_row_nnz", C.c_int), ("diag_min", C.c_double), ("diag_max", C.c_double), ("prec", C.c_int),
                ("prec_degree", C.c_int), ("prec_lmin", C.c_double), ("prec_lmax", C.c_double),
                ("format", C.c_int), ("dia_offsets", C.c_int)]


_lib = None


def load(path: str | None = None):
    """Load the built library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libsscg is not built ({p}); run __graft_entry__.build()")
    L = C.CDLL(p)
    vp, i64, i32, dbl, sz = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_size_t
    P = C.POINTER
    L.sscg_create.argtypes = [P(vp), vp]
    L.sscg_destroy.argtypes = [vp]
    L.sscg_last_error.argtypes = [vp]; L.sscg_last_error.restype = C.c_char_p
    L.sscg_status_str.argtypes = [i32]; L.sscg_status_str.restype = C.c_char_p
    L.sscg_mat_storage_bytes.argtypes = [i64, i64, P(sz)]
    L.sscg_mat_create_csr.argtypes = [vp, i64, i64, vp, vp, vp, C.c_uint, vp, sz, P(vp)]
    L.sscg_mat_destroy.argtypes = [vp]
    L.sscg_mat_props_get.argtypes = [vp, P(MatProps)]
    L.sscg_set_preconditioner.argtypes = [vp, i32, i32, dbl, dbl]
    L.sscg_solve_workspace_bytes.argtypes = [vp, P(Opts), P(sz)]
    L.sscg_solve.argtypes = [vp, vp, vp, vp, P(Opts), P(Info), vp, sz]
    L.sscg_pcg_workspace_bytes.argtypes = [vp, P(Opts), P(sz)]
    L.sscg_pcg_solve.argtypes = [vp, vp, vp, vp, P(Opts), P(Info), vp, sz]
    L.sscg_pfcg_workspace_bytes.argtypes = [vp, P(Opts), P(sz)]
    L.sscg_pfcg_solve.argtypes = [vp, vp, vp, vp, P(Opts), P(Info), vp, sz]
    L.sscg_spmv.argtypes = [vp, vp, vp, vp]
    L.sscg_bounds_workspace_bytes.argtypes = [vp, i32, P(sz)]
    L.sscg_estimate_bounds.argtypes = [vp, vp, i32, vp, vp, sz, P(dbl), P(dbl)]
    L.sscg_uniform.argtypes = [vp, i64, C.c_uint64, vp]
    L.sscg_solve_static.argtypes = [vp, vp, vp, vp, P(Opts), P(Info)]
    L.sscg_features_workspace_bytes.argtypes = [P(sz)]
    L.sscg_mat_features.argtypes = [vp, vp, vp, vp, sz]
    L.sscg_mlp_nparams.argtypes = [i32, i32, i32]; L.sscg_mlp_nparams.restype = i64
    L.sscg_mlp_workspace_bytes.argtypes = [i32, i32, i32, i32, P(sz)]
    L.sscg_mlp_forward.argtypes = [vp, i32, i32, i32, vp, i32, vp, vp, vp, sz]
    L.sscg_mlp_loss_grad.argtypes = [vp, i32, i32, i32, vp, i32, vp, vp, vp, P(dbl), vp, sz]
    L.sscg_mlp_adam_step.argtypes = [vp, i64, vp, vp, vp, vp, dbl, dbl, dbl, dbl, i32]
    L.sscg_mlp_train.argtypes = [vp, i32, i32, i32, vp, i32, vp, vp, i32, dbl, vp, vp, sz]
    L.sscg_bounds_mlp.argtypes = [vp, vp, i32, vp, vp, sz, P(dbl), P(dbl)]
    L.sscg_set_bounds_model.argtypes = [vp, i32, vp]
    L.sscg_batch_workspace_bytes.argtypes = [i32, vp, vp, P(Opts), P(sz)]
    L.sscg_batch_create.argtypes = [vp, i32, vp, vp, P(Opts), i32, vp, sz, P(vp)]
    L.sscg_batch_destroy.argtypes = [vp]
    L.sscg_batch_solve.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sscg_batch_props.argtypes = [vp, vp, P(i32), P(i32), P(C.c_float)]
    L.sscg_batch_launches.argtypes = [vp, P(C.c_int64)]
    L.sscg_probe_rate.argtypes = [vp, i32, i64, i64, P(dbl), P(dbl)]
    L.sscg_probe_small_solve.argtypes = [vp, i32, i32, P(dbl)]
    L.sscg_batch_inject_barrier_fault.argtypes = [vp, i32, i32]
    L.sscg_newton_shifts.argtypes = [i32, dbl, dbl, vp, P(dbl)]
    _lib = L
    return L


def newton_shifts(s, lmin, lmax):
    """(theta[0..s-2], sigma) of the solver's Newton basis over [lmin, lmax]
    (host-only; no GPU needed)."""
    L = load()
    theta = (C.c_double * max(s - 1, 1))()
    sig = C.c_double()
    rc = L.sscg_newton_shifts(int(s), float(lmin), float(lmax), theta, C.byref(sig))
    if rc != OK:
        raise SscgError(rc, "sscg_newton_shifts: invalid arguments")
    return np.array(theta[: s - 1]), sig.value


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("sscg needs a CUDA device; there is no CPU fallback")
    return torch


@dataclass
class SolveResult:
    status: int
    outer_iters: int
    equiv_iters: int
    rel_res_recursive: float
    rel_res_true: float
    hist: np.ndarray = field(default_factory=lambda: np.zeros(0))
    profile: dict = field(default_factory=dict)

    @property
    def converged(self) -> bool:
        return self.status == OK


class Context:
    """A library context bound to one CUDA stream (default: torch's current)."""

    def __init__(self, stream=None):
        torch = _torch()
        self.lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = self.lib.sscg_create(C.byref(h), C.c_void_p(self.stream.cuda_stream))
        if rc != OK:
            raise SscgError(rc, "sscg_create failed (no sm_103a device?)")
        self.h = h

    def uniform(self, n, seed):
        """Device U[-1, 1) vector: splitmix64 draws 0..n-1 from `seed`."""
        torch = _torch()
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        self.check(self.lib.sscg_uniform(self.h, n, seed, C.c_void_p(out.data_ptr())))
        return out

    def probe_rate(self, kind, iters_a, iters_b=0):
        """Throughput probe of include/sscg_probe.h: (operations per second
        over the device, kernel milliseconds)."""
        ops, ms = C.c_double(), C.c_double()
        self.check(self.lib.sscg_probe_rate(self.h, PROBE[kind], int(iters_a), int(iters_b), C.byref(ops),
                                            C.byref(ms)))
        return ops.value, ms.value

    def probe_small_solve(self, s, reps=100):
        """Latency probe of include/sscg_probe.h: mean SM cycles of the s x s
        Cholesky, the solves with 1 and with s right-hand sides, and the
        monomial step's first-step form."""
        out = (C.c_double * 4)()
        self.check(self.lib.sscg_probe_small_solve(self.h, int(s), int(reps), out))
        return dict(cholesky=out[0], solve_1=out[1], solve_s=out[2], monomial_step0=out[3])

    def check(self, rc, allow_positive=False):
        if rc < 0 or (rc > 0 and not allow_positive):
            raise SscgError(rc, self.lib.sscg_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.sscg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """CSR SPD matrix copied into torch-allocated device storage."""

    def __init__(self, ctx: Context, rowptr, col, val, csr_only=False):
        torch = _torch()
        self.ctx = ctx
        dev = torch.device("cuda", torch.cuda.current_device())

        def dev_tensor(a, dt):
            if isinstance(a, torch.Tensor):
                return a.to(device=dev, dtype=dt).contiguous()
            return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dt)

        rp = dev_tensor(rowptr, torch.int32)
        ci = dev_tensor(col, torch.int32)
        vv = dev_tensor(val, torch.float64)
        self.n = rp.numel() - 1
        self.nnz = ci.numel()
        nbytes = C.c_size_t()
        ctx.check(ctx.lib.sscg_mat_storage_bytes(self.n, self.nnz, C.byref(nbytes)))
        self.storage = torch.empty(nbytes.value, dtype=torch.uint8, device=dev)
        h = C.c_void_p()
        ctx.check(ctx.lib.sscg_mat_create_csr(ctx.h, self.n, self.nnz, C.c_void_p(rp.data_ptr()),
                                              C.c_void_p(ci.data_ptr()), C.c_void_p(vv.data_ptr()),
                                              MAT_CSR_ONLY if csr_only else 0,
                                              C.c_void_p(self.storage.data_ptr()), nbytes.value, C.byref(h)))
        self.h = h
        self.prec = "jacobi"

    def props(self) -> dict:
        p = MatProps()
        self.ctx.check(self.ctx.lib.sscg_mat_props_get(self.h, C.byref(p)))
        return {k: getattr(p, k) for k, _ in MatProps._fields_}

    def set_preconditioner(self, kind="jacobi", degree=0, lmin=0.0, lmax=0.0):
        self.ctx.check(self.ctx.lib.sscg_set_preconditioner(self.h, PREC[kind], int(degree), float(lmin), float(lmax)))
        self.prec = kind

    def estimate_bounds(self, steps=20, r0=None):
        """Extreme Ritz values of B^-1 A from `steps` Lanczos (CG) steps."""
        torch = _torch()
        nbytes = C.c_size_t()
        self.ctx.check(self.ctx.lib.sscg_bounds_workspace_bytes(self.h, steps, C.byref(nbytes)))
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.storage.device)
        lo, hi = C.c_double(), C.c_double()
        rp = C.c_void_p(r0.contiguous().data_ptr()) if r0 is not None else None
        self.ctx.check(self.ctx.lib.sscg_estimate_bounds(self.ctx.h, self.h, steps, rp, C.c_void_p(ws.data_ptr()),
                                                         nbytes.value, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def features(self):
        """The SSCG_NFEAT matrix features of the spectral-bound network (host array)."""
        torch = _torch()
        nbytes = C.c_size_t()
        self.ctx.check(self.ctx.lib.sscg_features_workspace_bytes(C.byref(nbytes)))
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.storage.device)
        f = torch.empty(NFEAT, dtype=torch.float64, device=self.storage.device)
        self.ctx.check(self.ctx.lib.sscg_mat_features(self.ctx.h, self.h, C.c_void_p(f.data_ptr()),
                                                      C.c_void_p(ws.data_ptr()), nbytes.value))
        return f.cpu().numpy()

    def bounds_mlp(self, hidden, model):
        """Spectral bounds of D^-1 A from a trained network; `model` is the
        device blob [x_mean, x_std, y_mean, y_std, theta] (FP64)."""
        torch = _torch()
        nbytes = C.c_size_t()
        self.ctx.check(self.ctx.lib.sscg_features_workspace_bytes(C.byref(nbytes)))
        ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.storage.device)
        lo, hi = C.c_double(), C.c_double()
        self.ctx.check(self.ctx.lib.sscg_bounds_mlp(self.ctx.h, self.h, int(hidden), C.c_void_p(model.data_ptr()),
                                                    C.c_void_p(ws.data_ptr()), nbytes.value, C.byref(lo),
                                                    C.byref(hi)))
        return lo.value, hi.value

    def set_bounds_model(self, hidden, model):
        """Attach a bounds network blob (kept alive here) for automatic
        Chebyshev-basis intervals; model=None detaches it."""
        rc = self.ctx.lib.sscg_set_bounds_model(self.h, int(hidden) if model is not None else 0,
                                                C.c_void_p(model.data_ptr()) if model is not None else None)
        if rc != OK:
            raise SscgError(rc, "sscg_set_bounds_model: bad width")
        self._bounds_model = model

    def spmv(self, x):
        torch = _torch()
        x = x.contiguous()
        y = torch.empty_like(x)
        self.ctx.check(self.ctx.lib.sscg_spmv(self.ctx.h, self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.sscg_mat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


DIRECT_GRAM = 0x4
FUSED_MPK = 0x8
ADAPTIVE_S = 0x20
FMA_UPDATE = 0x40


def make_opts(s=4, basis="monomial", tol=1e-8, maxit=1000, arith="f64", basis_bounds=(0.0, 0.0),
              replace_every=0, host_vectors=False, profile=False, direct_gram=False, fused_mpk=False,
              adaptive_s=False, fma_update=False) -> Opts:
    flags = (HOST_VECTORS if host_vectors else 0) | (PROFILE if profile else 0) | (DIRECT_GRAM if direct_gram else 0)
    flags |= (FUSED_MPK if fused_mpk else 0) | (ADAPTIVE_S if adaptive_s else 0) | (FMA_UPDATE if fma_update else 0)
    return Opts(int(s), BASIS[basis], float(basis_bounds[0]), float(basis_bounds[1]), float(tol), int(maxit),
                ARITH[arith], int(replace_every), flags)


class Solver:
    """Owns the workspace for repeated solves with one matrix and option set.
    method: "sstep" (Algorithm 3), "pcg" (Algorithm 1) or "pfcg" (Algorithm 2)."""

    def __init__(self, A: Matrix, method="sstep", **kw):
        torch = _torch()
        self.A = A
        self.method = method
        self.opts = make_opts(**kw)
        nbytes = C.c_size_t()
        lib = A.ctx.lib
        fn = {"sstep": lib.sscg_solve_workspace_bytes, "pcg": lib.sscg_pcg_workspace_bytes,
              "pfcg": lib.sscg_pfcg_workspace_bytes}[method]
        A.ctx.check(fn(A.h, C.byref(self.opts), C.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=A.storage.device)
        self.hist = np.zeros(self.opts.maxit + 2)

    def solve(self, b, x) -> SolveResult:
        """Solve in place: x holds x0 on entry and the solution on exit.
        b, x: FP64 device tensors, or host numpy/torch arrays when the solver
        was made with host_vectors=True."""
        ctx = self.A.ctx
        info = Info()
        info.hist = self.hist.ctypes.data_as(C.c_void_p).value
        info.hist_cap = len(self.hist)
        fn = {"sstep": ctx.lib.sscg_solve, "pcg": ctx.lib.sscg_pcg_solve, "pfcg": ctx.lib.sscg_pfcg_solve}[self.method]
        bp = b.ctypes.data if isinstance(b, np.ndarray) else b.data_ptr()
        xp = x.ctypes.data if isinstance(x, np.ndarray) else x.data_ptr()
        rc = fn(ctx.h, self.A.h, C.c_void_p(bp), C.c_void_p(xp), C.byref(self.opts), C.byref(info),
                C.c_void_p(self.workspace.data_ptr()), self.workspace.numel())
        ctx.check(rc, allow_positive=True)
        return SolveResult(info.status, info.outer_iters, info.equiv_iters, info.rel_res_recursive,
                           info.rel_res_true, self.hist[:info.hist_len].copy(),
                           {k: getattr(info, k) for k in _PROFILE_FIELDS})


def solve(A: Matrix, b, x=None, method="sstep", **kw):
    """One-shot convenience: returns (x, SolveResult)."""
    torch = _torch()
    if x is None:
        x = torch.zeros_like(b)
    r = Solver(A, method=method, **kw).solve(b, x)
    return x, r


@dataclass
class BatchResult:
    status: int
    systems: list          # SolveResult per system (worst over its right-hand sides)
    rhs: list              # SolveResult per right-hand side, systems in order
    latency_ms: np.ndarray  # device time until each system's result was final
    solve_ms: float         # CUDA-event time of the whole batched solve


class BatchSolver:
    """Plan for solving many systems (each with 1..8 right-hand sides) in one
    persistent launch; see sscg_batch_create."""

    def __init__(self, mats, nrhs, s=4, tol=1e-8, maxit=1000, arith="f64", tune=False, persistent=False,
                 fma_update=False):
        torch = _torch()
        self.mats = list(mats)
        self.nrhs = [int(r) for r in nrhs]
        assert len(self.mats) == len(self.nrhs)
        self.ctx = self.mats[0].ctx
        lib = self.ctx.lib
        k = len(self.mats)
        self._mh = (C.c_void_p * k)(*[m.h.value for m in self.mats])
        self._nr = (C.c_int * k)(*self.nrhs)
        self.opts = make_opts(s=s, tol=tol, maxit=maxit, arith=arith)
        if persistent:
            self.opts.flags |= BATCH_PERSISTENT
        if fma_update:
            self.opts.flags |= FMA_UPDATE
        nbytes = C.c_size_t()
        rc = lib.sscg_batch_workspace_bytes(k, self._mh, self._nr, C.byref(self.opts), C.byref(nbytes))
        if rc != OK:
            raise SscgError(rc, "sscg_batch_workspace_bytes: invalid batch")
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device="cuda")
        h = C.c_void_p()
        self.ctx.check(lib.sscg_batch_create(self.ctx.h, k, self._mh, self._nr, C.byref(self.opts), int(bool(tune)),
                                             C.c_void_p(self.workspace.data_ptr()), self.workspace.numel(),
                                             C.byref(h)))
        self.h = h

    def props(self):
        k = len(self.mats)
        tiles = (C.c_int * k)()
        grid, graph, ms = C.c_int(), C.c_int(), C.c_float()
        self.ctx.check(self.ctx.lib.sscg_batch_props(self.h, tiles, C.byref(grid), C.byref(graph), C.byref(ms)))
        nl = C.c_int64()
        self.ctx.check(self.ctx.lib.sscg_batch_launches(self.h, C.byref(nl)))
        return dict(tile_rows=list(tiles), grid=grid.value, graph=bool(graph.value), last_ms=ms.value,
                    launches=nl.value)

    def inject_barrier_fault(self, cta, wait_ms):
        """Arm the next solve of a persistent plan: CTA `cta` skips its first
        grid-barrier arrival and barrier waits give up after wait_ms (the
        solve then returns TIMEOUT); cta=-1 disarms."""
        self.ctx.check(self.ctx.lib.sscg_batch_inject_barrier_fault(self.h, int(cta), int(wait_ms)))

    def solve(self, B, X) -> BatchResult:
        """B[k], X[k]: FP64 device tensors of shape (nrhs[k], n_k) (each
        right-hand side contiguous); X holds x0 and receives the solution."""
        k = len(self.mats)
        for i in range(k):
            assert B[i].is_contiguous() and X[i].is_contiguous()
            assert tuple(B[i].shape) == (self.nrhs[i], self.mats[i].n) == tuple(X[i].shape)
        bp = (C.c_void_p * k)(*[t.data_ptr() for t in B])
        xp = (C.c_void_p * k)(*[t.data_ptr() for t in X])
        infos = (Info * k)()
        rinf = (Info * sum(self.nrhs))()
        lat = np.zeros(k)
        rc = self.ctx.lib.sscg_batch_solve(self.h, bp, xp, infos, rinf, lat.ctypes.data_as(C.c_void_p))
        self.ctx.check(rc, allow_positive=True)

        def res(i):
            return SolveResult(i.status, i.outer_iters, i.equiv_iters, i.rel_res_recursive, i.rel_res_true)

        return BatchResult(rc, [res(i) for i in infos], [res(i) for i in rinf], lat, self.props()["last_ms"])

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.sscg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
