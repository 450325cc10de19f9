"""Host-side checks of the C-ABI boundary (no GPU needed): the library builds for sm_103a,
loads, and exports every entry point that include/helm.h declares; the binding rejects bad
arguments before any device work."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "helm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(?:helm_status\s+|void\s+|const char\s*\*\s*)(\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("helm_create", "helm_apply", "mg_vcycle", "krylov_solve", "helm_solve_adjoint",
                     "helm_grad_k2", "helm_create_batch", "helm_solve_batch", "helm_destroy",
                     "helm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1012_4307_gb300 import build
    path = build.build()
    import ctypes
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a():
    from paper_1012_4307_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    path = build.build()
    data = open(path, "rb").read()
    assert b"sm_103a" in data or b"sm_103" in data


def test_version_and_error_strings_without_gpu():
    import ctypes as C
    from paper_1012_4307_gb300 import helm
    lib = helm.load()
    assert "sm_103a" in helm.helm_version()
    assert isinstance(helm.helm_last_error(), str)
    # a null handle is rejected before any device work
    assert lib.helm_apply(None, 0, 0, None, None) == helm.HELM_ERR_ARG
    assert "null" in helm.helm_last_error()
    assert lib.krylov_solve(None, 0, None, None, 1e-8, 30, 10, None) == helm.HELM_ERR_ARG
    assert lib.mg_vcycle(None, None, None, 0) == helm.HELM_ERR_ARG
    assert lib.mg_precondition(None, None, None, 0) == helm.HELM_ERR_ARG
    t = helm._Tuning()
    assert lib.helm_set_tuning(None, C.byref(t)) == helm.HELM_ERR_ARG
    assert lib.helm_get_tuning(None, C.byref(t)) == helm.HELM_ERR_ARG
    assert lib.helm_autotune(None, 1, 10, None, None) == helm.HELM_ERR_ARG


def test_create_rejects_bad_arguments_without_gpu():
    import ctypes as C
    from paper_1012_4307_gb300 import helm
    lib = helm.load()
    g = helm._Grid()
    g.dim = 4
    mg = helm.MGParams().to_c()
    out = C.c_void_p()
    r = (C.c_double * 3)(-0.75, -0.75, -0.75)
    st = lib.helm_create(C.byref(g), 0.5, r, r, C.c_void_p(16), C.byref(mg), None, C.byref(out))
    assert st == helm.HELM_ERR_ARG and "dim" in helm.helm_last_error()
    g.dim, g.n[0], g.n[1] = 2, 17, 17
    g.lo[0] = g.lo[1] = -1.0
    g.hi[0] = g.hi[1] = 1.0
    mg.omega = 3.0
    st = lib.helm_create(C.byref(g), 0.5, r, r, C.c_void_p(16), C.byref(mg), None, C.byref(out))
    assert st == helm.HELM_ERR_ARG and "omega" in helm.helm_last_error()
    mg = helm.MGParams(kind="qd", re_lambda0=0.0).to_c()
    st = lib.helm_create(C.byref(g), 0.5, r, r, C.c_void_p(16), C.byref(mg), None, C.byref(out))
    assert st == helm.HELM_ERR_ARG and "QD" in helm.helm_last_error()
