"""Adjoint gradient at the full adjoint workload: L = |sum g u|^2 for a Gaussian probe g on the
513 x 513 ECS grid (k^2 = 2(E - V), E = 2, growth toward the boundary), u = A(k^2)^{-1} f with a
complex64 V-cycle inside FP64 FGMRES.  torch.autograd through HelmholtzSolve (adjoint solve
A^T lambda = conj(dL/du) by A^T = W A W^{-1}, then dL/dk^2 = Re(lambda u)) against central
differences of L along 8 seeded smooth directions (Gaussian bumps of k^2 in the real region):
the directional derivative sum_p grad_p d_p must match (L(k^2 + eps d) - L(k^2 - eps d)) / 2 eps.
A bump moves L far above the solver's residual floor, so the difference quotient is clean; a
single-node perturbation of k^2 at this size would not be.  dL/dV = -2 dL/dk^2."""
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
    tol = 2e-12  # the FP64 true residual bottoms out near 4e-13 at this size

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
    rng = np.random.default_rng(2024)
    centres = rng.integers(n // 4, 3 * n // 4, size=(8, 2))  # interior (real) region
    yy, xx = np.mgrid[0:n, 0:n]
    eps = 1e-4
    fds, dds = [], []
    for (cj, ci) in centres:
        d = np.exp(-((xx - ci) ** 2 + (yy - cj) ** 2) / (2.0 * 6.0 ** 2))
        vals = []
        for sgn in (1, -1):
            h = factory(torch.from_numpy(P.k2 + sgn * eps * d))
            uu, st = helm.krylov_solve(h, f, tol=tol, restart=30, maxit=6000)
            assert st.status == helm.HELM_OK
            vals.append(float(((g * uu).sum().abs() ** 2).item()))
            h.close()
        fds.append((vals[0] - vals[1]) / (2 * eps))
        dds.append(float((grad * d).sum()))
    fds, dds = np.array(fds), np.array(dds)
    # normwise over the directions: central-difference truncation O(eps^2) and solve noise
    # (relative residual 2e-12) both sit well below 1e-4 of the largest directional derivative
    err = np.abs(fds - dds).max()
    assert err <= 1e-4 * np.abs(dds).max(), (err, fds.tolist(), dds.tolist())


def test_adjoint_gradient_513_pointwise(helm):
    """Central differences at 32 seeded single nodes of the same 513 x 513 problem.  A step of
    1e-6 at one node moves L by about 1e-10 of itself at this size, below what a solve to a
    relative residual of 1e-12 resolves, so the step is 1e-2 (k^2 is about 14 in the real
    region): L then moves by about 1e-6 of itself while the O(step^2) truncation stays far below
    the 1e-4 normwise bound."""
    P = W.config_adjoint(513)
    n = P.n
    g = to_gpu(P.extra["probe"]).to(torch.complex128)
    f = to_gpu(P.f)
    tol = 2e-12

    def factory(k2):
        Pk = W.Problem("adj", 2, n, k2.cpu().numpy(), P.f, coarsest_n=17)
        return gpu_handle(helm, Pk, pc="csg", prec="c64", gs="fp64")

    k2 = to_gpu(P.k2).requires_grad_(True)
    u = helm.HelmholtzSolve.apply(k2, f, factory, tol, 30, 6000)
    L = (g * u).sum().abs() ** 2
    L.backward()
    grad = k2.grad.cpu().numpy()
    rng = np.random.default_rng(2025)
    idx = rng.integers(n // 4, 3 * n // 4, size=(32, 2))
    step = 1e-2
    fds, gps = [], []
    for (j, i) in idx:
        vals = []
        for sgn in (1, -1):
            kk = P.k2.copy()
            kk[j, i] += sgn * step
            h = factory(torch.from_numpy(kk))
            uu, st = helm.krylov_solve(h, f, tol=tol, restart=30, maxit=6000)
            assert st.status == helm.HELM_OK
            vals.append(float(((g * uu).sum().abs() ** 2).item()))
            h.close()
        fds.append((vals[0] - vals[1]) / (2 * step))
        gps.append(grad[j, i])
    fds, gps = np.array(fds), np.array(gps)
    err = np.abs(fds - gps).max()
    assert err <= 1e-4 * np.abs(gps).max(), (err, fds.tolist(), gps.tolist())
