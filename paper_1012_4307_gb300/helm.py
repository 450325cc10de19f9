"""Python binding of libhelm.so (argument marshalling only; all arithmetic runs in the
library's sm_103a kernels).

The functions carry the C-ABI names of ``include/helm.h``: :func:`helm_create`,
:func:`helm_apply`, :func:`mg_vcycle`, :func:`krylov_solve`, :func:`helm_solve_adjoint`,
:func:`helm_grad_k2`, :func:`helm_mg_conv`, :func:`helm_create_batch`,
:func:`helm_solve_batch`.  Vectors are CUDA torch tensors holding every grid node including
the Dirichlet boundary (shape ``(n1, n0)`` or ``(n2, n1, n0)``, x fastest), complex128 for
HELM_C128 and complex64 for HELM_C64.  PyTorch provides device memory and the stream; there is
no CPU fallback: without the library or a GPU every call raises.

:class:`HelmholtzSolve` is a ``torch.autograd.Function`` whose backward solves the adjoint
system A^T lambda = conj(grad_u) with the same operator and preconditioner
(A^T = W A W^{-1}, W the complex dual-volume weights of the FD scheme), then forms
dL/dk^2 = Re(lambda * u) in the library.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass, field

import torch

from . import build as _build

HELM_OK, HELM_ERR_ARG, HELM_ERR_CUDA, HELM_ERR_NOMEM, HELM_ERR_NOCONV, HELM_ERR_BREAKDOWN, \
    HELM_ERR_NONFINITE, HELM_ERR_TIMEOUT = range(8)
HELM_C128, HELM_C64 = 0, 1
HELM_PC_NONE, HELM_PC_CSG, HELM_PC_CSL, HELM_PC_QD, HELM_PC_LAPLACE = range(5)
HELM_OP_A, HELM_OP_M = 0, 1
HELM_FGMRES, HELM_BICGSTAB = 0, 1
HELM_SMOOTH_JACOBI, HELM_SMOOTH_RB = 0, 1
HELM_GS_FP64, HELM_GS_DF, HELM_GS_DCGS2 = 0, 1, 2

PC_KINDS = {"none": HELM_PC_NONE, "csg": HELM_PC_CSG, "csl": HELM_PC_CSL, "qd": HELM_PC_QD, "laplace": HELM_PC_LAPLACE}
STATUS_NAMES = {0: "HELM_OK", 1: "HELM_ERR_ARG", 2: "HELM_ERR_CUDA", 3: "HELM_ERR_NOMEM", 4: "HELM_ERR_NOCONV",
                5: "HELM_ERR_BREAKDOWN", 6: "HELM_ERR_NONFINITE", 7: "HELM_ERR_TIMEOUT"}


class HelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class _MG(C.Structure):
    _fields_ = [("kind", C.c_int), ("theta_a", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("re_lambda0", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double),
                ("smoother", C.c_int), ("gamma_f", C.c_int), ("gamma_c", C.c_int), ("coarsest_n", C.c_int),
                ("prec", C.c_int), ("gs_arith", C.c_int)]


HELM_MAX_LEVELS = 16
TILES = {"none": -1, "32x8": 0, "16x16": 1, "16x8": 2, "64x4": 3, "wave": 4, "8x8": 5}
_TILE_NAMES = {v: k for k, v in TILES.items()}


class _Tuning(C.Structure):
    _fields_ = [("tail_levels", C.c_int), ("level_tile", C.c_int * HELM_MAX_LEVELS),
                ("cluster_levels", C.c_int), ("cluster_ctas", C.c_int), ("cluster_halo", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("status", C.c_int), ("rel_res", C.c_double),
                ("est_res", C.c_double), ("time_ms", C.c_double), ("history", C.c_void_p),
                ("history_len", C.c_int), ("reorthogonalizations", C.c_int)]


_lock = threading.Lock()
_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Loads libhelm.so (building it first if its sources are newer).  Raises if unavailable."""
    global _LIB
    with _lock:
        if _LIB is not None:
            return _LIB
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libhelm.so is not built (%s); run paper_1012_4307_gb300.build.build()" % path)
        lib = C.CDLL(path)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        sigs = {
            "helm_create": ([P, D, P, P, P, P, P, P], I),
            "helm_destroy": ([P], None),
            "helm_apply": ([P, I, I, P, P], I),
            "mg_vcycle": ([P, P, P, I], I),
            "mg_precondition": ([P, P, P, I], I),
            "krylov_solve": ([P, I, P, P, D, I, I, P], I),
            "helm_solve_adjoint": ([P, P, P, D, I, I, P], I),
            "helm_grad_k2": ([P, P, P, P], I),
            "helm_backward": ([P, P, P, P, P, D, I, I, P], I),
            "helm_qd_lambda0": ([P, D, P, P, P, I, P], I),
            "helm_mg_conv": ([P, P, P, I, D, I, P, P], I),
            "helm_mg_conv_noalloc": ([P, P, P, I, D, I, P, P], I),
            "helm_levels": ([P, P], I),
            "helm_level_shape": ([P, I, P], I),
            "helm_create_batch": ([I, P, P, P, P, P, P, P], I),
            "helm_solve_batch": ([P, P, P, D, I, I, P], I),
            "helm_destroy_batch": ([P], None),
            "helm_batch_handle": ([P, I, P], I),
            "helm_batch_set_engine": ([P, I], I),
            "helm_batch_get_engine": ([P, P], I),
            "helm_profile": ([P, I], I),
            "helm_set_tuning": ([P, P], I),
            "helm_get_tuning": ([P, P], I),
            "helm_autotune": ([P, I, I, P, P], I),
            "helm_profile_read": ([P, I, P, P, P, P, P], I),
            "helm_last_error": ([], C.c_char_p),
            "helm_version": ([], C.c_char_p),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = lib
        return lib


def helm_last_error() -> str:
    return load().helm_last_error().decode()


def helm_version() -> str:
    return load().helm_version().decode()


def _check(st, allow=(HELM_OK,)):
    if st not in allow:
        raise HelmError(st, helm_last_error())
    return st


@dataclass
class MGParams:
    """Mirror of ``helm_mg_params`` (Section 4.2, Algorithm 1, Section 5 operators)."""
    kind: str = "csg"
    theta_a: float = math.pi / 14
    beta1: float = -1.0
    beta2: float = -0.5
    re_lambda0: float = 0.0
    nu1: int = 2
    nu2: int = 2
    omega: float = 0.8
    smoother: str = "jacobi"
    gamma_f: int = 1
    gamma_c: int = 1
    coarsest_n: int = 17
    prec: str = "c64"
    # Arnoldi arithmetic: "fp64" (IEEE FP64, CGS + DGKS), "df" (double-FP32 on float-pair
    # vectors, CGS + DGKS) or "dcgs2" (double-FP32, delayed CGS2: one dot and one update pass)
    gs: str = "fp64"

    def to_c(self) -> _MG:
        m = _MG()
        m.kind = PC_KINDS[self.kind]
        m.theta_a, m.beta1, m.beta2, m.re_lambda0 = self.theta_a, self.beta1, self.beta2, self.re_lambda0
        m.nu1, m.nu2, m.omega = self.nu1, self.nu2, self.omega
        m.smoother = HELM_SMOOTH_RB if self.smoother == "rb" else HELM_SMOOTH_JACOBI
        m.gamma_f, m.gamma_c, m.coarsest_n = self.gamma_f, self.gamma_c, self.coarsest_n
        m.prec = HELM_C64 if self.prec == "c64" else HELM_C128
        m.gs_arith = {"fp64": HELM_GS_FP64, "df": HELM_GS_DF, "dcgs2": HELM_GS_DCGS2}[self.gs]
        return m


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _vec(t: torch.Tensor, np_: int, name: str, dtype=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if not t.is_contiguous() or t.numel() != np_:
        raise ValueError("%s must be contiguous with %d elements" % (name, np_))
    return t.data_ptr()


def _prec_of(t: torch.Tensor) -> int:
    if t.dtype == torch.complex128:
        return HELM_C128
    if t.dtype == torch.complex64:
        return HELM_C64
    raise TypeError("grid vectors must be complex128 or complex64 (got %s)" % t.dtype)


class Handle:
    """Owns one ``helm_handle*`` (solver for one grid, its levels and workspace)."""

    def __init__(self, ptr, dim, n, stream, owned=True):
        self.ptr = ptr
        self.dim = dim
        self.n = tuple(n[:dim])
        self.shape = tuple(reversed(self.n))
        self.np = int(math.prod(self.n))
        self.stream = stream
        self.owned = owned

    def __del__(self):
        if getattr(self, "ptr", None) and _LIB is not None and self.owned:
            _LIB.helm_destroy(self.ptr)
        self.ptr = None

    def close(self):
        self.__del__()

    @property
    def levels(self):
        n = C.c_int()
        _check(load().helm_levels(self.ptr, C.byref(n)))
        out = []
        for l in range(n.value):
            s = (C.c_int * 3)()
            _check(load().helm_level_shape(self.ptr, l, s))
            out.append(tuple(reversed(list(s)[: self.dim])))
        return out

    def zeros(self, dtype=torch.complex128):
        return torch.zeros(self.shape, dtype=dtype, device="cuda")


def helm_create(dim, n, k2: torch.Tensor, theta=math.pi / 6, r0_lo=None, r0_hi=None, lo=None, hi=None,
                mg: MGParams | None = None, stream=None) -> Handle:
    """helm_create(): ECS grid, operator A = -Delta - k^2, preconditioner hierarchy."""
    n = list(n) if hasattr(n, "__len__") else [n] * dim
    lo = list(lo) if lo is not None else [-1.0] * dim
    hi = list(hi) if hi is not None else [1.0] * dim
    r0_lo = list(r0_lo) if r0_lo is not None else [-0.75] * dim
    r0_hi = list(r0_hi) if r0_hi is not None else [0.75] * dim
    mg = mg or MGParams()
    g = _Grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = n[a] if a < dim else 1
        g.lo[a] = lo[a] if a < dim else 0.0
        g.hi[a] = hi[a] if a < dim else 1.0
    npts = int(math.prod(n[:dim]))
    k2 = k2.to(device="cuda", dtype=torch.float64).contiguous()
    ptr_k2 = _vec(k2, npts, "k2", torch.float64)
    rl = (C.c_double * 3)(*(r0_lo + [0.0] * (3 - dim)))
    rh = (C.c_double * 3)(*(r0_hi + [0.0] * (3 - dim)))
    out = C.c_void_p()
    mgc = mg.to_c()
    _check(load().helm_create(C.byref(g), float(theta), rl, rh, C.c_void_p(ptr_k2), C.byref(mgc),
                              _stream_ptr(stream), C.byref(out)))
    h = Handle(out.value, dim, n, stream)
    h.mg = mg
    return h


def helm_qd_lambda0(dim, n, k2_axis, theta=math.pi / 6, r0_lo=None, r0_hi=None, lo=None, hi=None,
                    mode: str = "axes") -> float:
    """Re(lambda0) for the QD preconditioner from per-axis k^2 profiles (host computation in the
    library): mode "axes" = the one-dimensional counterpart (exact for a separable k^2 field),
    "max_k2" = minus the largest k^2.  k2_axis: dim 1D arrays of n[a] values at the real nodes."""
    import numpy as np
    n = list(n) if hasattr(n, "__len__") else [n] * dim
    lo = list(lo) if lo is not None else [-1.0] * dim
    hi = list(hi) if hi is not None else [1.0] * dim
    r0_lo = list(r0_lo) if r0_lo is not None else [-0.75] * dim
    r0_hi = list(r0_hi) if r0_hi is not None else [0.75] * dim
    g = _Grid()
    g.dim = dim
    for a in range(3):
        g.n[a] = n[a] if a < dim else 1
        g.lo[a] = lo[a] if a < dim else 0.0
        g.hi[a] = hi[a] if a < dim else 1.0
    prof = [np.ascontiguousarray(k2_axis[a], dtype=np.float64) for a in range(dim)]
    for a in range(dim):
        if prof[a].shape != (n[a],):
            raise ValueError("k2_axis[%d] must hold %d values" % (a, n[a]))
    ptrs = (C.c_void_p * 3)(*([p.ctypes.data for p in prof] + [None] * (3 - dim)))
    rl = (C.c_double * 3)(*(r0_lo + [0.0] * (3 - dim)))
    rh = (C.c_double * 3)(*(r0_hi + [0.0] * (3 - dim)))
    out = C.c_double()
    _check(load().helm_qd_lambda0(C.byref(g), float(theta), rl, rh, ptrs, {"axes": 0, "max_k2": 1}[mode],
                                  C.byref(out)))
    return out.value


def helm_destroy(h: Handle):
    h.close()


def helm_apply(h: Handle, x: torch.Tensor, y: torch.Tensor | None = None, which: str = "A") -> torch.Tensor:
    """y = A x (which='A') or y = M x (which='M'), in the precision of x."""
    prec = _prec_of(x)
    if y is None:
        y = torch.zeros_like(x)
    _check(load().helm_apply(h.ptr, HELM_OP_A if which == "A" else HELM_OP_M, prec,
                             C.c_void_p(_vec(x, h.np, "x")), C.c_void_p(_vec(y, h.np, "y", x.dtype))))
    return y


def mg_vcycle(h: Handle, b: torch.Tensor, x: torch.Tensor | None = None) -> torch.Tensor:
    """One cycle of Algorithm 1 for M x = b; x is the initial guess (zero if None), updated in place."""
    prec = _prec_of(b)
    if x is None:
        x = torch.zeros_like(b)
    _check(load().mg_vcycle(h.ptr, C.c_void_p(_vec(b, h.np, "b")), C.c_void_p(_vec(x, h.np, "x", b.dtype)), prec))
    return x


def mg_precondition(h: Handle, v: torch.Tensor, dtype: torch.dtype = torch.complex64) -> torch.Tensor:
    """The outer solvers' preconditioner call: one cycle from zero for M z = v (v complex128,
    z of the given dtype, complex64 = the cycle in complex64)."""
    if v.dtype != torch.complex128:
        raise TypeError("v must be complex128")
    z = torch.zeros(v.shape, dtype=dtype, device=v.device)
    prec = _prec_of(z)
    _check(load().mg_precondition(h.ptr, C.c_void_p(_vec(v, h.np, "v")), C.c_void_p(_vec(z, h.np, "z", dtype)), prec))
    return z


@dataclass
class Stats:
    iterations: int = 0
    restarts: int = 0
    status: int = 0
    rel_res: float = float("nan")
    est_res: float = float("nan")
    time_ms: float = 0.0
    history: list = field(default_factory=list)
    reorthogonalizations: int = 0


def _stats_from(s: _Stats, hist) -> Stats:
    out = Stats(s.iterations, s.restarts, s.status, s.rel_res, s.est_res, s.time_ms)
    out.reorthogonalizations = s.reorthogonalizations
    if hist is not None:
        out.history = list(hist[: min(s.iterations, len(hist))])
    return out


def krylov_solve(h: Handle, rhs: torch.Tensor, x: torch.Tensor | None = None, tol=1e-8, restart=30, maxit=1000,
                 method: str = "fgmres", history: bool = False, raise_on_noconv: bool = True):
    """Solves A x = rhs (FP64) with FGMRES(restart) or Bi-CGSTAB; returns (x, Stats)."""
    if x is None:
        x = torch.zeros_like(rhs)
    hist = (C.c_double * maxit)() if history else None
    st = _Stats()
    if hist is not None:
        st.history = C.cast(hist, C.c_void_p)
        st.history_len = maxit
    allow = (HELM_OK,) if raise_on_noconv else (HELM_OK, HELM_ERR_NOCONV)
    _check(load().krylov_solve(h.ptr, HELM_BICGSTAB if method == "bicgstab" else HELM_FGMRES,
                               C.c_void_p(_vec(rhs, h.np, "rhs", torch.complex128)),
                               C.c_void_p(_vec(x, h.np, "x", torch.complex128)), float(tol), int(restart),
                               int(maxit), C.byref(st)), allow)
    return x, _stats_from(st, hist)


def helm_solve_adjoint(h: Handle, rhs: torch.Tensor, tol=1e-8, restart=30, maxit=1000, raise_on_noconv=True):
    lam = torch.zeros_like(rhs)
    st = _Stats()
    allow = (HELM_OK,) if raise_on_noconv else (HELM_OK, HELM_ERR_NOCONV)
    _check(load().helm_solve_adjoint(h.ptr, C.c_void_p(_vec(rhs, h.np, "rhs", torch.complex128)),
                                     C.c_void_p(_vec(lam, h.np, "lambda", torch.complex128)), float(tol),
                                     int(restart), int(maxit), C.byref(st)), allow)
    return lam, _stats_from(st, None)


def helm_grad_k2(h: Handle, lam: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    grad = torch.empty(h.shape, dtype=torch.float64, device="cuda")
    _check(load().helm_grad_k2(h.ptr, C.c_void_p(_vec(lam, h.np, "lambda", torch.complex128)),
                               C.c_void_p(_vec(u, h.np, "u", torch.complex128)), C.c_void_p(grad.data_ptr())))
    return grad


def helm_backward(h: Handle, grad_u: torch.Tensor, u: torch.Tensor | None, grad_k2: torch.Tensor | None,
                  grad_f: torch.Tensor | None, tol=1e-10, restart=30, maxit=2000, raise_on_noconv=True):
    """Adjoint step in the library: solves A^T lambda = conj(grad_u) and writes
    grad_k2 = Re(lambda u) and grad_f = conj(lambda) into the given tensors (either may be None)."""
    st = _Stats()
    allow = (HELM_OK,) if raise_on_noconv else (HELM_OK, HELM_ERR_NOCONV)
    pk2 = C.c_void_p(_vec(grad_k2, h.np, "grad_k2", torch.float64)) if grad_k2 is not None else None
    pf = C.c_void_p(_vec(grad_f, h.np, "grad_f", torch.complex128)) if grad_f is not None else None
    pu = C.c_void_p(_vec(u, h.np, "u", torch.complex128)) if u is not None else None
    _check(load().helm_backward(h.ptr, C.c_void_p(_vec(grad_u, h.np, "grad_u", torch.complex128)), pu, pk2, pf,
                                float(tol), int(restart), int(maxit), C.byref(st)), allow)
    return _stats_from(st, None)


def helm_mg_conv(h: Handle, b: torch.Tensor, tol=1e-6, maxcyc=100):
    """Stand-alone multigrid (Section 5 "mg-conv"): returns (x, cycles, factor)."""
    x = torch.zeros_like(b)
    nc, fac = C.c_int(), C.c_double()
    _check(load().helm_mg_conv(h.ptr, C.c_void_p(_vec(b, h.np, "b")), C.c_void_p(_vec(x, h.np, "x", b.dtype)),
                               _prec_of(b), float(tol), int(maxcyc), C.byref(nc), C.byref(fac)))
    return x, nc.value, fac.value


KERNEL_CLASSES = ["apply", "smooth_fine", "smooth_coarse", "restrict", "prolong", "coarse", "mdot",
                  "update_mdot", "update_norm", "vector", "small"]


def helm_profile(h: Handle, enable: bool = True):
    """Reset and enable (or disable) per-launch CUDA-event timing on the handle's stream."""
    _check(load().helm_profile(h.ptr, 1 if enable else 0))


def helm_profile_read(h: Handle) -> dict:
    """Per kernel class: launches, summed event time (ms), algorithmic bytes and flops, and the
    bytes counted pass by pass (bytes_pass)."""
    nc = len(KERNEL_CLASSES)
    la, ms, by, fl, bp = ((C.c_int * nc)(), (C.c_double * nc)(), (C.c_double * nc)(), (C.c_double * nc)(),
                          (C.c_double * nc)())
    _check(load().helm_profile_read(h.ptr, nc, la, ms, by, fl, bp))
    return {name: dict(launches=la[i], ms=ms[i], bytes=by[i], flops=fl[i], bytes_pass=bp[i])
            for i, name in enumerate(KERNEL_CLASSES)}


def _tuning_to_dict(t: _Tuning, nlev: int) -> dict:
    return {"tail_levels": t.tail_levels, "level_tile": [_TILE_NAMES[t.level_tile[l]] for l in range(nlev)],
            "cluster_levels": t.cluster_levels, "cluster_ctas": t.cluster_ctas, "cluster_halo": t.cluster_halo}


def helm_get_tuning(h: Handle) -> dict:
    """The handle's kernel choices: tail_levels (-1 = as many as fit), a tile name per level
    ("none" = separate sweep / residual / transfer launches), cluster_levels (0 = off),
    cluster_ctas (8 or 16) and cluster_halo (1 or 3 rows beyond each block's slab)."""
    t = _Tuning()
    _check(load().helm_get_tuning(h.ptr, C.byref(t)))
    return _tuning_to_dict(t, len(h.levels))


def helm_set_tuning(h: Handle, tuning: dict):
    t = _Tuning()
    _check(load().helm_get_tuning(h.ptr, C.byref(t)))
    t.tail_levels = int(tuning.get("tail_levels", t.tail_levels))
    for l, name in enumerate(tuning.get("level_tile", [])[:HELM_MAX_LEVELS]):
        t.level_tile[l] = TILES[name]
    t.cluster_levels = int(tuning.get("cluster_levels", t.cluster_levels))
    t.cluster_ctas = int(tuning.get("cluster_ctas", t.cluster_ctas))
    t.cluster_halo = int(tuning.get("cluster_halo", t.cluster_halo))
    _check(load().helm_set_tuning(h.ptr, C.byref(t)))


def tuning_key(h: Handle, prec: str) -> str:
    """Cache key of a tuning: everything the choice depends on (grid, levels, cycle, precision)."""
    mg = getattr(h, "mg", None) or MGParams()
    return "%dd-%s-%s-%s-nu%d%d-g%d%d-c%d-%s" % (h.dim, "x".join(map(str, h.n)), mg.kind, mg.smoother, mg.nu1, mg.nu2,
                                                  mg.gamma_f, mg.gamma_c, mg.coarsest_n, prec)


def default_tuning_cache() -> str:
    """A cache file beside the built library, named by the library's content hash (a rebuilt
    library starts a new cache)."""
    import hashlib
    with open(_build.LIB, "rb") as fh:
        tag = hashlib.sha1(fh.read()).hexdigest()[:12]
    return os.path.join(os.path.dirname(_build.LIB), "tuning-%s.json" % tag)


def cached_tuning(h: Handle, prec: str = "c64", cache: str | None = None):
    """The stored tuning for this handle's key, or None."""
    import json
    cache = cache or default_tuning_cache()
    if not os.path.exists(cache):
        return None
    with open(cache) as fh:
        return json.load(fh).get(tuning_key(h, prec), {}).get("tuning")


def helm_autotune(h: Handle, prec: str = "c64", reps: int = 25, cache: str | None = None, retune: bool = False):
    """Picks the cycle's kernels (tail depth, tile shape per level) by timing preconditioner
    applications on the device, installs the choice and returns (tuning dict, ms per cycle).
    With a cache path (JSON, keyed by tuning_key), a stored choice is installed without timing
    unless retune; new results are stored."""
    import json
    key = tuning_key(h, prec)
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            table = json.load(fh)
        if key in table and not retune:
            helm_set_tuning(h, table[key]["tuning"])
            return table[key]["tuning"], table[key]["ms"]
    t, ms = _Tuning(), C.c_double()
    _check(load().helm_autotune(h.ptr, HELM_C64 if prec == "c64" else HELM_C128, int(reps), C.byref(t), C.byref(ms)))
    tuning = _tuning_to_dict(t, len(h.levels))
    if cache:
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        table[key] = {"tuning": tuning, "ms": ms.value}
        tmp = cache + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return tuning, ms.value


def helm_mg_conv_noalloc(h: Handle, b: torch.Tensor, x: torch.Tensor, tol=1e-6, maxcyc=100):
    """helm_mg_conv computed in the library's fixed scratch array (no allocation at all, not
    even here: the caller passes the output ``x``).  For callers that cannot allocate at the
    point of the call: a service whose device memory is sized once at start-up, or a loop that
    cannot afford the device-wide synchronisation an allocation may cause.  Returns (cycles,
    factor); x is overwritten with the stand-alone multigrid iterate."""
    nc, fac = C.c_int(), C.c_double()
    _check(load().helm_mg_conv_noalloc(h.ptr, C.c_void_p(_vec(b, h.np, "b")), C.c_void_p(_vec(x, h.np, "x", b.dtype)),
                                       _prec_of(b), float(tol), int(maxcyc), C.byref(nc), C.byref(fac)))
    return nc.value, fac.value


class Batch:
    def __init__(self, ptr, shapes):
        self.ptr = ptr
        self.shapes = shapes

    def __del__(self):
        if getattr(self, "ptr", None) and _LIB is not None:
            _LIB.helm_destroy_batch(self.ptr)
            self.ptr = None


def helm_create_batch(problems, mg: MGParams | None = None, stream=None) -> Batch:
    """problems: list of dicts with dim, n, k2 (CUDA float64 tensor), theta, r0_lo, r0_hi, lo, hi."""
    mg = mg or MGParams()
    nb = len(problems)
    grids = (_Grid * nb)()
    theta = (C.c_double * nb)()
    r0 = (C.c_double * (6 * nb))()
    k2p = (C.c_void_p * nb)()
    keep = []
    shapes = []
    for i, p in enumerate(problems):
        dim = p["dim"]
        n = list(p["n"]) if hasattr(p["n"], "__len__") else [p["n"]] * dim
        grids[i].dim = dim
        for a in range(3):
            grids[i].n[a] = n[a] if a < dim else 1
            grids[i].lo[a] = p.get("lo", [-1.0] * dim)[a] if a < dim else 0.0
            grids[i].hi[a] = p.get("hi", [1.0] * dim)[a] if a < dim else 1.0
            r0[6 * i + a] = p.get("r0_lo", [-0.75] * dim)[a] if a < dim else 0.0
            r0[6 * i + 3 + a] = p.get("r0_hi", [0.75] * dim)[a] if a < dim else 0.0
        theta[i] = p.get("theta", math.pi / 6)
        k2 = p["k2"].to(device="cuda", dtype=torch.float64).contiguous()
        keep.append(k2)
        k2p[i] = k2.data_ptr()
        shapes.append(tuple(reversed(n[:dim])))
    out = C.c_void_p()
    mgc = mg.to_c()
    _check(load().helm_create_batch(nb, grids, theta, r0, k2p, C.byref(mgc), _stream_ptr(stream), C.byref(out)))
    bt = Batch(out.value, shapes)
    bt.mg = mg
    return bt


def batch_handle(b: Batch, i: int) -> Handle:
    """Problem i's handle, owned by the batch (valid while the batch lives)."""
    out = C.c_void_p()
    _check(load().helm_batch_handle(b.ptr, int(i), C.byref(out)))
    shape = b.shapes[i]
    h = Handle(out.value, len(shape), list(reversed(shape)), None, owned=False)
    h.mg = b.mg
    h._batch = b
    return h


def helm_autotune_batch(b: Batch, prec: str = "c64", reps: int = 25, cache: str | None = None) -> dict:
    """Autotunes one handle per distinct grid of the batch (through helm_autotune and its cache)
    and installs the choice on every problem with that grid; returns {tuning key: tuning}."""
    chosen = {}
    for i in range(len(b.shapes)):
        h = batch_handle(b, i)
        key = tuning_key(h, prec)
        if key not in chosen:
            chosen[key], _ = helm_autotune(h, prec, reps=reps, cache=cache)
        else:
            helm_set_tuning(h, chosen[key])
    return chosen


BATCH_ENGINES = {"auto": 0, "lockstep": 1, "streams": 2}
_BATCH_ENGINE_NAMES = {v: k for k, v in BATCH_ENGINES.items()}


def helm_batch_set_engine(b: Batch, engine: str):
    """Engine of helm_solve_batch: "lockstep" (every phase of a step one launch over all
    problems), "streams" (one stream per problem) or "auto" (lockstep when it applies)."""
    _check(load().helm_batch_set_engine(b.ptr, BATCH_ENGINES[engine]))


def helm_batch_get_engine(b: Batch) -> str:
    """The engine the last helm_solve_batch ran ("auto" before any)."""
    e = C.c_int()
    _check(load().helm_batch_get_engine(b.ptr, C.byref(e)))
    return _BATCH_ENGINE_NAMES[e.value]


def helm_solve_batch(b: Batch, rhs, x, tol=1e-8, restart=30, maxit=1000, raise_on_noconv=True):
    nb = len(b.shapes)
    rp = (C.c_void_p * nb)(*[_vec(r, int(math.prod(s)), "rhs", torch.complex128) for r, s in zip(rhs, b.shapes)])
    xp = (C.c_void_p * nb)(*[_vec(v, int(math.prod(s)), "x", torch.complex128) for v, s in zip(x, b.shapes)])
    st = (_Stats * nb)()
    allow = (HELM_OK,) if raise_on_noconv else (HELM_OK, HELM_ERR_NOCONV)
    _check(load().helm_solve_batch(b.ptr, rp, xp, float(tol), int(restart), int(maxit), st), allow)
    return [_stats_from(s, None) for s in st]


class HelmholtzSolve(torch.autograd.Function):
    """u = A(k^2)^{-1} f with A = -Delta - k^2 (ECS, FP64 FGMRES, multigrid preconditioner).

    forward(k2, f, handle_factory, tol, restart, maxit) -> u.  ``handle_factory(k2)`` returns
    a :class:`Handle` for that k^2.  Only u is saved (the Krylov basis is not kept).  backward
    is one library call (helm_backward): it solves A^T lambda = conj(grad_u) by the adjoint
    identity and writes dL/dk^2 = Re(lambda u) and dL/df = conj(lambda) (PyTorch passes
    grad_u = 2 dL/d(conj u) for a real loss L).
    """

    @staticmethod
    def forward(ctx, k2, f, handle_factory, tol=1e-10, restart=30, maxit=2000):
        h = handle_factory(k2.detach())
        u, st = krylov_solve(h, f.detach().contiguous(), tol=tol, restart=restart, maxit=maxit)
        ctx.h = h
        ctx.opts = (tol, restart, maxit)
        ctx.save_for_backward(u)
        ctx.stats = st
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        tol, restart, maxit = ctx.opts
        # marshalling only: complex128, contiguous, and a lazily conjugated view materialised
        # (the library reads the memory as it is)
        gu = grad_u.to(torch.complex128).resolve_conj().contiguous()
        g = torch.empty(u.shape, dtype=torch.float64, device=u.device) if ctx.needs_input_grad[0] else None
        gf = torch.empty_like(u) if ctx.needs_input_grad[1] else None
        if g is not None or gf is not None:
            helm_backward(ctx.h, gu, u, g, gf, tol=tol, restart=restart, maxit=maxit)
        return g, gf, None, None, None, None
