"""Adjoint gradient at the full adjoint workload: L = |sum g u|^2 for a Gaussian probe g on the
513 x 513 ECS grid (k^2 = 2(E - V), E = 2, growth toward the boundary), u = A(k^2)^{-1} f with a
complex64 V-cycle inside FP64 FGMRES.  torch.autograd through HelmholtzSolve (adjoint solve
A^T lambda = conj(dL/du) by A^T = W A W^{-1}, then dL/dk^2 = Re(lambda u)) against central
differences with step 1e-6 at 32 seeded points; dL/dV = -2 dL/dk^2."""
import numpy as np
import pytest

from helpers import gpu_handle, to_gpu
from paper_1012_4307_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_4307_gb300 import helm as H
    H.load()
    return H


def test_adjoint_gradient_513_central_differences(helm):
    P = W.config_adjoint(513)
    n = P.n
    g = to_gpu(P.extra["probe"]).to(torch.complex128)
    f = to_gpu(P.f)
    tol = 1e-13

    def factory(k2):
        Pk = W.Problem("adj", 2, n, k2.cpu().numpy(), P.f, coarsest_n=17)
        return gpu_handle(helm, Pk, pc="csg", prec="c64", gs="fp64")

    k2 = to_gpu(P.k2).requires_grad_(True)
    u = helm.HelmholtzSolve.apply(k2, f, factory, tol, 30, 6000)
    L = (g * u).sum().abs() ** 2
    L.backward()
    grad = k2.grad.cpu().numpy()
    gmax = np.abs(grad).max()
    assert np.isfinite(gmax) and gmax > 0
    # dL/dV = -2 dL/dk^2 since k^2 = 2 (E - V)
    rng = np.random.default_rng(2024)
    idx = rng.integers(n // 4, 3 * n // 4, size=(32, 2))  # interior (real) region
    errs = []
    for (j, i) in idx:
        vals = []
        for sgn in (1, -1):
            kk = P.k2.copy()
            kk[j, i] += sgn * 1e-6
            h = factory(torch.from_numpy(kk))
            uu, st = helm.krylov_solve(h, f, tol=tol, restart=30, maxit=6000)
            vals.append(float(((g * uu).sum().abs() ** 2).item()))
            h.close()
        fd = (vals[0] - vals[1]) / 2e-6
        errs.append(abs(fd - grad[j, i]))
    # normwise relative gradient error (the difference quotient carries ~tol * L / step of noise)
    assert max(errs) <= 1e-5 * gmax, (max(errs), gmax)
