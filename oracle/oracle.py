"""Python front end of the plain FP64 CPU oracle (helm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The GPU library never imports or calls it, and it imports
nothing from the GPU package.

What it computes is stated in helm_oracle.c, function by function, with the passage of the
paper (bin Zubair, Reps, Vanroose, arXiv 1012.4307) each follows:

* ``contour``          -- the ECS contour z(x) with a linear scaling function (Section 3.1).
* ``Op.apply``         -- M = a L_h(widths * e^{i ts}) + bk k^2 + c, where L_h is the
                          non-uniform three-point FD negative Laplacian (Section 3.2).
* ``Op.jacobi / rb``   -- omega-Jacobi and omega-red-black Jacobi (Section 4.2).
* ``restrict / prolong_add`` -- full weighting and bi/trilinear interpolation (Section 4.2).
* ``MG.cycle``         -- the recursion MG(l, A, b, u, nu1, nu2, C, gamma_f, gamma_c)
                          (Algorithm 1) on rediscretised levels.
* ``fgmres / bicgstab``-- the outer Krylov solvers (Sections 5 and 6).
* ``helmholtz_ops``    -- the operators A = Z = -Delta - k^2 and the preconditioners
                          M_CSL, M_CSG, M_QD and the Laplacian of Section 5.

Arrays are numpy, C-ordered with x fastest: shape (n0,), (n1, n0) or (n2, n1, n0), including
the Dirichlet boundary nodes (kept at zero).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "helm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
# The same source built with -fopenmp: independent node loops shared out over the host's cores
# (reductions stay serial, so every result is bit-identical to the single-threaded build).
# Selected by HELM_ORACLE_OPENMP=1 in the environment before the first call; used only for the
# all-cores CPU baseline.
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None


def _compile(out: str, extra) -> None:
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False, openmp: bool | None = None) -> str:
    """Compile helm_oracle.c with gcc (FP64, no contraction of a*b+c into FMAs), single-threaded
    and with -fopenmp; returns the path of the variant in use."""
    os.makedirs(_BUILD, exist_ok=True)
    for path, extra in ((_LIB_PATH, []), (_LIB_OMP_PATH, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            _compile(path, extra)
    if openmp is None:
        openmp = os.environ.get("HELM_ORACLE_OPENMP", "0") == "1"
    return _LIB_OMP_PATH if openmp else _LIB_PATH


def threads() -> int:
    """Threads the loaded oracle uses (1 for the single-threaded build)."""
    if os.environ.get("HELM_ORACLE_OPENMP", "0") != "1":
        return 1
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


class _COp(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("z", C.c_void_p * 3),
                ("a", C.c_double * 2), ("bk", C.c_double * 2), ("c", C.c_double * 2),
                ("ts", C.c_double), ("k2", C.c_void_p)]


class _CStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("rel_res", C.c_double), ("history", C.c_void_p), ("history_len", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.or_contour.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, P]
            for name in ("or_apply", "or_apply_T", "or_residual"):
                getattr(lib, name).restype = None
            lib.or_apply.argtypes = [P, P, P]
            lib.or_apply_T.argtypes = [P, P, P]
            lib.or_diag.argtypes = [P, P]
            lib.or_weights.argtypes = [P, P]
            lib.or_residual.argtypes = [P, P, P, P]
            lib.or_jacobi.argtypes = [P, C.c_double, C.c_int, P, P]
            lib.or_rbjacobi.argtypes = [P, C.c_double, C.c_int, P, P]
            lib.or_restrict.argtypes = [C.c_int, P, P, P]
            lib.or_prolong_add.argtypes = [C.c_int, P, P, P]
            lib.or_lu_factor.argtypes = [C.c_int, P, P]
            lib.or_lu_factor.restype = C.c_int
            lib.or_lu_solve.argtypes = [C.c_int, P, P, P]
            lib.or_mg_create.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int]
            lib.or_mg_create.restype = P
            lib.or_mg_destroy.argtypes = [P]
            lib.or_mg_levels.argtypes = [P]
            lib.or_mg_levels.restype = C.c_int
            lib.or_mg_level_shape.argtypes = [P, C.c_int, P]
            lib.or_mg_ok.argtypes = [P]
            lib.or_mg_ok.restype = C.c_int
            lib.or_mg_cycle.argtypes = [P, P, P, C.c_int, C.c_int]
            lib.or_fgmres.argtypes = [P, P, C.c_int, C.c_int, P, P, C.c_double, C.c_int, C.c_int, P]
            lib.or_fgmres.restype = C.c_int
            lib.or_bicgstab.argtypes = [P, P, C.c_int, C.c_int, P, P, C.c_double, C.c_int, P]
            lib.or_bicgstab.restype = C.c_int
            lib.or_mg_conv.argtypes = [P, C.c_int, C.c_int, P, C.c_double, C.c_int, P, P]
            lib.or_mg_conv.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def contour(n: int, lo: float, hi: float, theta: float, r0lo: float, r0hi: float) -> np.ndarray:
    """Complex ECS nodes of one axis (Section 3.1); a side with r0 beyond the domain has no layer."""
    z = np.zeros(n, dtype=np.complex128)
    _load().or_contour(n, lo, hi, theta, r0lo, r0hi, _ptr(z))
    return z


class Op:
    """M = a L_h(widths e^{i ts}) + bk diag(k^2) + c on the complex nodes ``z`` (one array per axis)."""

    def __init__(self, z, k2, a=1.0, bk=-1.0, c=0.0, ts=0.0):
        self.dim = len(z)
        self.z = [_c128(zz) for zz in z]
        self.n = [len(zz) for zz in self.z] + [1] * (3 - self.dim)
        self.shape = tuple(reversed(self.n[: self.dim]))
        self.k2 = np.ascontiguousarray(np.broadcast_to(np.asarray(k2, dtype=np.float64), self.shape))
        self.a, self.bk, self.c, self.ts = complex(a), complex(bk), complex(c), float(ts)
        s = _COp()
        s.dim = self.dim
        for i in range(3):
            s.n[i] = self.n[i]
            s.z[i] = _ptr(self.z[i]) if i < self.dim else _ptr(self.z[0])
        s.a[0], s.a[1] = self.a.real, self.a.imag
        s.bk[0], s.bk[1] = self.bk.real, self.bk.imag
        s.c[0], s.c[1] = self.c.real, self.c.imag
        s.ts = self.ts
        s.k2 = _ptr(self.k2)
        self._s = s

    @property
    def ref(self):
        return C.byref(self._s)

    def _vec(self, x):
        x = _c128(x)
        assert x.shape == self.shape, (x.shape, self.shape)
        return x

    def apply(self, x):
        x = self._vec(x)
        y = np.empty_like(x)
        _load().or_apply(self.ref, _ptr(x), _ptr(y))
        return y

    def apply_T(self, x):
        x = self._vec(x)
        y = np.empty_like(x)
        _load().or_apply_T(self.ref, _ptr(x), _ptr(y))
        return y

    def diag(self):
        d = np.empty(self.shape, dtype=np.complex128)
        _load().or_diag(self.ref, _ptr(d))
        return d

    def weights(self):
        w = np.empty(self.shape, dtype=np.complex128)
        _load().or_weights(self.ref, _ptr(w))
        return w

    def residual(self, f, u):
        f, u = self._vec(f), self._vec(u)
        r = np.empty_like(f)
        _load().or_residual(self.ref, _ptr(f), _ptr(u), _ptr(r))
        return r

    def jacobi(self, f, u, omega, sweeps=1):
        f, u = self._vec(f), self._vec(u).copy()
        _load().or_jacobi(self.ref, omega, sweeps, _ptr(f), _ptr(u))
        return u

    def rbjacobi(self, f, u, omega, sweeps=1):
        f, u = self._vec(f), self._vec(u).copy()
        _load().or_rbjacobi(self.ref, omega, sweeps, _ptr(f), _ptr(u))
        return u

    def interior_mask(self):
        m = np.zeros(self.shape, dtype=bool)
        m[(slice(1, -1),) * self.dim] = True
        return m

    def dense(self):
        """Dense matrix on the interior unknowns, assembled column by column from ``apply``."""
        mask = self.interior_mask().ravel()
        idx = np.flatnonzero(mask)
        A = np.zeros((idx.size, idx.size), dtype=np.complex128)
        e = np.zeros(self.shape, dtype=np.complex128)
        ef = e.reshape(-1)
        for c, p in enumerate(idx):
            ef[p] = 1.0
            A[:, c] = self.apply(e).reshape(-1)[idx]
            ef[p] = 0.0
        return A


def restrict(rf: np.ndarray) -> np.ndarray:
    rf = _c128(rf)
    dim = rf.ndim
    nf = (C.c_int * 3)(*(list(reversed(rf.shape)) + [1] * (3 - dim)))
    rc = np.empty(tuple((s + 1) // 2 for s in rf.shape), dtype=np.complex128)
    _load().or_restrict(dim, C.byref(nf), _ptr(rf), _ptr(rc))
    return rc


def prolong_add(ec: np.ndarray, uf: np.ndarray) -> np.ndarray:
    ec, uf = _c128(ec), _c128(uf).copy()
    dim = uf.ndim
    nf = (C.c_int * 3)(*(list(reversed(uf.shape)) + [1] * (3 - dim)))
    assert ec.shape == tuple((s + 1) // 2 for s in uf.shape)
    _load().or_prolong_add(dim, C.byref(nf), _ptr(ec), _ptr(uf))
    return uf


def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Textbook LU with partial pivoting on a dense complex matrix."""
    n = A.shape[0]
    LU = np.asfortranarray(A, dtype=np.complex128).copy(order="F")
    piv = np.zeros(n, dtype=np.int32)
    if _load().or_lu_factor(n, LU.ctypes.data, piv.ctypes.data) != 0:
        raise np.linalg.LinAlgError("singular")
    x = _c128(b).copy()
    _load().or_lu_solve(n, LU.ctypes.data, piv.ctypes.data, x.ctypes.data)
    return x


class MG:
    """Rediscretised multigrid hierarchy for ``op`` (Section 4.2) and Algorithm 1's cycle."""

    def __init__(self, op: Op, coarsest_n: int, nu1=2, nu2=2, omega=0.8, smoother="jacobi"):
        self.op = op
        self.h = _load().or_mg_create(op.ref, coarsest_n, nu1, nu2, omega, 1 if smoother == "rb" else 0)
        if not _load().or_mg_ok(self.h):
            raise np.linalg.LinAlgError("singular coarsest operator")

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.or_mg_destroy(h)
            self.h = None

    @property
    def nlev(self):
        return _load().or_mg_levels(self.h)

    def level_shape(self, l):
        n = (C.c_int * 3)()
        _load().or_mg_level_shape(self.h, l, C.byref(n))
        return tuple(reversed(list(n)[: self.op.dim]))

    def cycle(self, b, u=None, gamma_f=1, gamma_c=1):
        b = self.op._vec(b)
        u = np.zeros_like(b) if u is None else self.op._vec(u).copy()
        _load().or_mg_cycle(self.h, _ptr(b), _ptr(u), gamma_f, gamma_c)
        return u

    def mg_conv(self, b, tol=1e-6, maxcyc=100, gamma_f=1, gamma_c=1):
        b = self.op._vec(b)
        fac = C.c_double()
        hist = np.zeros(maxcyc)
        ncyc = _load().or_mg_conv(self.h, gamma_f, gamma_c, _ptr(b), tol, maxcyc, C.byref(fac), _ptr(hist))
        return ncyc, fac.value, hist[:ncyc]


def _solve(kind, A: Op, mg, f, x0, tol, restart, maxit, gamma_f, gamma_c, history):
    f = A._vec(f)
    x = np.zeros_like(f) if x0 is None else A._vec(x0).copy()
    hist = np.zeros(max(maxit, 1))
    st = _CStats()
    st.history = _ptr(hist) if history else None
    st.history_len = hist.size if history else 0
    mgh = mg.h if mg is not None else None
    if kind == "fgmres":
        _load().or_fgmres(A.ref, mgh, gamma_f, gamma_c, _ptr(f), _ptr(x), tol, restart, maxit, C.byref(st))
    else:
        _load().or_bicgstab(A.ref, mgh, gamma_f, gamma_c, _ptr(f), _ptr(x), tol, maxit, C.byref(st))
    stats = dict(iterations=st.iterations, restarts=st.restarts, status=st.status, rel_res=st.rel_res)
    if history:
        stats["history"] = hist[: st.iterations].copy()
    return x, stats


def fgmres(A: Op, mg, f, x0=None, tol=1e-10, restart=30, maxit=1000, gamma_f=1, gamma_c=1, history=False):
    """Right-preconditioned flexible GMRES(restart) with one MG cycle as preconditioner."""
    return _solve("fgmres", A, mg, f, x0, tol, restart, maxit, gamma_f, gamma_c, history)


def bicgstab(A: Op, mg, f, x0=None, tol=1e-10, maxit=1000, gamma_f=1, gamma_c=1, history=False):
    """Right-preconditioned Bi-CGSTAB, two MG cycles per iteration (Section 5)."""
    return _solve("bicgstab", A, mg, f, x0, tol, 0, maxit, gamma_f, gamma_c, history)


# ---------------------------------------------------------------------------------------
# The model problem and the preconditioning operators of Section 5.

def axes(dim, n, lo=-1.0, hi=1.0, theta=math.pi / 6, r0lo=-0.75, r0hi=0.75):
    """Complex nodes of every axis: the same ECS contour on each axis (Section 3.1)."""
    return [contour(n, lo, hi, theta, r0lo, r0hi) for _ in range(dim)]


def helmholtz_ops(z, k2, pc="csg", theta_a=math.pi / 14, beta=(-1.0, -0.5), re_lambda0=None):
    """A = Z = L_h - k^2 (eq. 2.1 with l1 = l2 = 0, discretised as in Section 3.2), and the
    preconditioning operator of Section 5:

    * ``csl``: M = L_h + (beta1 + i beta2) k^2  (complex-shifted Laplacian);
    * ``csg``: M = Z on the grid whose widths are multiplied by e^{i theta_a};
    * ``qd``:  M = (1 - i) I + Z / |Re lambda0|  (quadrant-definite, eq. 4.1 in table form);
    * ``laplace``: M = L_h;  ``none``: no preconditioner.
    """
    A = Op(z, k2, a=1.0, bk=-1.0, c=0.0, ts=0.0)
    if pc == "none":
        return A, None
    if pc == "csl":
        M = Op(z, k2, a=1.0, bk=complex(beta[0], beta[1]), c=0.0)
    elif pc == "csg":
        M = Op(z, k2, a=1.0, bk=-1.0, c=0.0, ts=theta_a)
    elif pc == "qd":
        s = 1.0 / abs(re_lambda0)
        M = Op(z, k2, a=s, bk=-s, c=1.0 - 1.0j)
    elif pc == "laplace":
        M = Op(z, k2, a=1.0, bk=0.0, c=0.0)
    else:
        raise ValueError(pc)
    return A, M
