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


def test_backward_against_dense_torch_autograd(helm, oracle):
    """helm_backward (one library call: adjoint solve, dL/dk^2 and dL/df on the device) against
    PyTorch's own reverse mode through a dense LU solve on the CPU, at 17 x 17 nodes: the same
    loss L = |sum g u|^2 differentiated with respect to k^2 and to the (complex) source f."""
    from helpers import oracle_pair, small_problem_adjoint
    P = small_problem_adjoint(17)
    n = P.n
    A, _ = oracle_pair(oracle, P)
    k2i = P.k2[1:-1, 1:-1].ravel()
    Lh = torch.from_numpy(A.dense() + np.diag(k2i))          # L_h = A + diag(k^2)
    g = torch.from_numpy(W.gaussian_source(2, n, 0.1, 78).real.copy())
    # reference: dense solve on the interior unknowns, PyTorch autograd on the CPU
    k2_ref = torch.from_numpy(k2i.copy()).requires_grad_(True)
    f_ref = torch.from_numpy(P.f[1:-1, 1:-1].ravel().copy()).requires_grad_(True)
    u_ref = torch.linalg.solve(Lh - torch.diag(k2_ref.to(torch.complex128)), f_ref)
    L_ref = (g[1:-1, 1:-1].reshape(-1).to(torch.complex128) * u_ref).sum().abs() ** 2
    L_ref.backward()

    def factory(k2):
        P2 = W.Problem("t", 2, n, k2.cpu().numpy(), P.f, coarsest_n=17)
        return gpu_handle(helm, P2, pc="csg", prec="c128")

    k2 = to_gpu(P.k2).requires_grad_(True)
    f = to_gpu(P.f).requires_grad_(True)
    u = helm.HelmholtzSolve.apply(k2, f, factory, 1e-13, 30, 2000)
    L = (g.cuda().to(u.dtype) * u).sum().abs() ** 2
    L.backward()
    gk = k2.grad.cpu().numpy()
    gf = f.grad.cpu().numpy()
    rk = k2_ref.grad.numpy()
    rf = f_ref.grad.numpy()
    assert np.abs(gk[1:-1, 1:-1].ravel() - rk).max() <= 1e-9 * np.abs(rk).max()
    assert np.abs(gf[1:-1, 1:-1].ravel() - rf).max() <= 1e-9 * np.abs(rf).max()
    # boundary entries are zero
    assert np.all(gk[0, :] == 0) and np.all(gf[:, 0] == 0)


def test_adjoint_gradient_129_against_oracle(helm, oracle):
    """dL/dk^2 at 129 x 129 nodes (between the dense check and the finite differences at 513)
    against a gradient computed entirely by the oracle: u from its FGMRES, lambda from its
    FGMRES on A with the right-hand side W^{-1} conj(grad_u) multiplied back by its dual-volume
    weights W, confirmed by its own transposed operator (||A^T lambda - conj(grad_u)|| small),
    and Re(lambda u).  Both sides solve to 1e-12; the gradients agree to 1e-8 (relative l2)."""
    from helpers import oracle_pair, small_problem_adjoint
    P = small_problem_adjoint(129)
    n = P.n
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, 17, 2, 2, 0.8)
    g = W.gaussian_source(2, n, 0.05, 79).real.copy()
    uo, st = oracle.fgmres(A, mg, P.f, tol=1e-12, restart=30, maxit=3000)
    assert st["status"] == 0
    s = np.sum(g * uo)
    grad_u = 2.0 * s * g  # what reverse mode hands backward for L = |sum g u|^2 with g real
    rhs = np.conj(grad_u)
    w = A.weights()
    inner = np.zeros_like(rhs)
    inner[1:-1, 1:-1] = rhs[1:-1, 1:-1] / w[1:-1, 1:-1]
    yo, st = oracle.fgmres(A, mg, inner, tol=1e-12, restart=30, maxit=3000)
    assert st["status"] == 0
    lam = w * yo
    lam[0, :] = lam[-1, :] = lam[:, 0] = lam[:, -1] = 0
    res = A.apply_T(lam) - rhs
    assert np.linalg.norm(res[1:-1, 1:-1]) <= 1e-10 * np.linalg.norm(rhs)
    ref = np.zeros(P.k2.shape)
    ref[1:-1, 1:-1] = np.real(lam * uo)[1:-1, 1:-1]

    def factory(k2):
        P2 = W.Problem("t", 2, n, k2.cpu().numpy(), P.f, coarsest_n=17)
        return gpu_handle(helm, P2, pc="csg", prec="c128")

    k2 = to_gpu(P.k2).requires_grad_(True)
    u = helm.HelmholtzSolve.apply(k2, to_gpu(P.f), factory, 1e-12, 30, 3000)
    L = (to_gpu(g).to(u.dtype) * u).sum().abs() ** 2
    L.backward()
    grad = k2.grad.cpu().numpy()
    err = np.linalg.norm(grad - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err
