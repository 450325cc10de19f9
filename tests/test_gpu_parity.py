"""CUDA path against the CPU oracle on identical seeded inputs (element by element, relative
l2 over the whole node array).  Tolerances: stencil apply 1e-14, one multigrid cycle 1e-12, the
FP64 solution 1e-8 at a relative residual of 1e-10 (FP64 paths); complex64 paths are checked
against FP32 rounding bounds and their FP64-outer residual guarantee."""
import math

import numpy as np
import pytest

from helpers import gpu_handle, oracle_pair, rel_l2, to_gpu, to_np
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


def small_problem(dim, n, seed=0, kh=0.5, E=2.0):
    P = W.Problem("t", dim, n, W.k2_well_growth(dim, n, E=E, kh_max=kh), W.gaussian_source(dim, n, 0.1, seed),
                  coarsest_n=17 if dim == 2 else 9)
    return P


# ---------------------------------------------------------------------------- stencil apply

@pytest.mark.parametrize("dim,n", [(2, 5), (2, 17), (2, 33), (2, 65), (2, 129), (2, 97), (3, 5), (3, 9), (3, 17), (3, 33)])
@pytest.mark.parametrize("which,pc", [("A", "csg"), ("M", "csg"), ("M", "csl"), ("M", "qd"), ("M", "laplace")])
def test_apply_c128(helm, oracle, dim, n, which, pc):
    P = small_problem(dim, n)
    kw = dict(re_lambda0=-123.0) if pc == "qd" else {}
    h = gpu_handle(helm, P, pc=pc, **kw)
    A, M = oracle_pair(oracle, P, pc=pc, **({"re_lambda0": -123.0} if pc == "qd" else {}))
    op = A if which == "A" else M
    x = W.random_field(P.k2.shape, 100 + n)
    y = helm.helm_apply(h, to_gpu(x), which=which)
    ref = op.apply(x)
    assert rel_l2(to_np(y), ref) <= 1e-14


@pytest.mark.parametrize("dim,n", [(2, 65), (2, 33), (3, 17)])
def test_apply_c64(helm, oracle, dim, n):
    P = small_problem(dim, n)
    h = gpu_handle(helm, P, pc="csg")
    A, M = oracle_pair(oracle, P, pc="csg")
    x = W.random_field(P.k2.shape, 7).astype(np.complex64)
    for which, op in (("A", A), ("M", M)):
        y = helm.helm_apply(h, to_gpu(x), which=which)
        assert rel_l2(to_np(y), op.apply(x.astype(np.complex128))) <= 2e-6


def test_apply_leaves_boundary_untouched(helm):
    P = small_problem(2, 33)
    h = gpu_handle(helm, P)
    x = to_gpu(W.random_field(P.k2.shape, 3))
    y = torch.full_like(x, 7 + 7j)
    helm.helm_apply(h, x, y)
    yy = to_np(y)
    assert np.all(yy[0, :] == 7 + 7j) and np.all(yy[-1, :] == 7 + 7j)
    assert np.all(yy[:, 0] == 7 + 7j) and np.all(yy[:, -1] == 7 + 7j)


def test_nonsquare_grid(helm, oracle):
    n = [65, 33]
    k2 = W.k2_constant(2, 65, 8.0)[:33, :]
    f = np.zeros((33, 65), complex)
    f[1:-1, 1:-1] = W.random_field((33, 65), 4)[1:-1, 1:-1]
    P = W.Problem("ns", 2, n, k2, f, coarsest_n=17)
    h = gpu_handle(helm, P)
    A, M = oracle_pair(oracle, P)
    x = W.random_field((33, 65), 9)
    assert rel_l2(to_np(helm.helm_apply(h, to_gpu(x))), A.apply(x)) <= 1e-14
    mg = oracle.MG(M, 17, 2, 2, 0.8, "jacobi")
    assert h.levels == [mg.level_shape(l) for l in range(mg.nlev)]
    assert rel_l2(to_np(helm.mg_vcycle(h, to_gpu(f))), mg.cycle(f)) <= 1e-12


# ---------------------------------------------------------------------------- one cycle

CYCLES = [
    dict(dim=2, n=65, pc="csg", smoother="jacobi", nu=(2, 2), omega=0.8, gamma=(1, 1)),
    dict(dim=2, n=33, pc="csl", smoother="jacobi", nu=(1, 1), omega=0.5, gamma=(1, 2)),
    dict(dim=2, n=65, pc="qd", smoother="rb", nu=(1, 1), omega=1.05, gamma=(1, 1)),
    dict(dim=2, n=65, pc="csg", smoother="jacobi", nu=(1, 1), omega=0.8, gamma=(1, 3)),
    dict(dim=2, n=33, pc="laplace", smoother="rb", nu=(2, 1), omega=1.0, gamma=(2, 2)),
    dict(dim=2, n=129, pc="csg", smoother="jacobi", nu=(2, 2), omega=0.8, gamma=(1, 1)),
    dict(dim=3, n=17, pc="csg", smoother="jacobi", nu=(2, 2), omega=0.8, gamma=(1, 1)),
    dict(dim=3, n=33, pc="csl", smoother="rb", nu=(1, 1), omega=1.0, gamma=(1, 2)),
]


@pytest.mark.parametrize("cfg", CYCLES, ids=lambda c: "%dd-n%d-%s-%s-%s" % (c["dim"], c["n"], c["pc"], c["smoother"], c["gamma"]))
@pytest.mark.parametrize("guess", ["zero", "random"])
def test_cycle_c128(helm, oracle, cfg, guess):
    P = small_problem(cfg["dim"], cfg["n"])
    kw = dict(re_lambda0=-200.0) if cfg["pc"] == "qd" else {}
    h = gpu_handle(helm, P, pc=cfg["pc"], smoother=cfg["smoother"], nu=cfg["nu"], omega=cfg["omega"],
                   gamma=cfg["gamma"], **kw)
    A, M = oracle_pair(oracle, P, pc=cfg["pc"], **kw)
    mg = oracle.MG(M, P.coarsest_n, cfg["nu"][0], cfg["nu"][1], cfg["omega"], cfg["smoother"])
    b = W.random_field(P.k2.shape, 11)
    u0 = W.random_field(P.k2.shape, 12) if guess == "random" else np.zeros_like(b)
    x = helm.mg_vcycle(h, to_gpu(b), to_gpu(u0))
    ref = mg.cycle(b, u0, *cfg["gamma"])
    assert rel_l2(to_np(x), ref) <= 1e-12


@pytest.mark.parametrize("dim,n", [(2, 65), (3, 17)])
def test_cycle_c64_close_to_fp64(helm, oracle, dim, n):
    P = small_problem(dim, n)
    h = gpu_handle(helm, P, pc="csg")
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, P.coarsest_n, 2, 2, 0.8, "jacobi")
    b = W.random_field(P.k2.shape, 21)
    x = helm.mg_vcycle(h, to_gpu(b.astype(np.complex64)))
    assert rel_l2(to_np(x), mg.cycle(b)) <= 1e-5


PRECOND_CASES = [(2, 65), (2, 97), (2, 129), (2, 257), (2, 1025), (2, (129, 65)), (3, 33)]


@pytest.mark.parametrize("dim,n", PRECOND_CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_precondition_matches_oracle(helm, oracle, dim, n, prec):
    """The outer solvers' preconditioner call (one cycle from zero on a complex128 vector).  On
    2D complex64 grids with V(2,2) omega-Jacobi this runs the temporally blocked kernels (two
    sweeps + residual + full weighting per tile, and prolongation + two sweeps per tile)."""
    if isinstance(n, tuple):
        nx, ny = n
        k2 = W.k2_well_growth(2, nx, kh_max=0.5)[:ny, :]
        f = np.zeros((ny, nx), complex)
        P = W.Problem("pc", 2, [nx, ny], k2, f, coarsest_n=17)
        shape = (ny, nx)
    else:
        P = small_problem(dim, n)
        shape = P.k2.shape
    h = gpu_handle(helm, P, pc="csg", prec=prec)
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, P.coarsest_n, 2, 2, 0.8, "jacobi")
    v = W.random_field(shape, 31)
    z = to_np(helm.mg_precondition(h, to_gpu(v), torch.complex64 if prec == "c64" else torch.complex128))
    ref = mg.cycle(v)
    tol = 1e-12 if prec == "c128" else 2e-5
    assert rel_l2(z, ref) <= tol
    # boundary nodes untouched (zero)
    assert np.all(z[..., 0] == 0) and np.all(z[..., -1] == 0)


def test_single_level_is_exact_solve(helm, oracle):
    P = small_problem(2, 9)
    h = gpu_handle(helm, P, pc="csl", coarsest_n=9)
    assert len(h.levels) == 1
    A, M = oracle_pair(oracle, P, pc="csl")
    b = W.random_field(P.k2.shape, 5)
    x = to_np(helm.mg_vcycle(h, to_gpu(b)))
    ref = np.zeros_like(b)
    ref[1:-1, 1:-1] = np.linalg.solve(M.dense(), b[1:-1, 1:-1].ravel()).reshape(7, 7)
    assert rel_l2(x, ref) <= 1e-12


# ---------------------------------------------------------------------------- Krylov solves

def test_fgmres_fp64_matches_oracle(helm, oracle):
    """Config: 2D 65 x 65 nodes, constant k = 10, ECS at pi/6 beyond 0.75, Gaussian source,
    CSG V(2,2) omega-Jacobi 0.8, GMRES(30) to 1e-10, all FP64."""
    P = W.config_small(65)
    h = gpu_handle(helm, P, pc="csg", prec="c128")
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, 17, 2, 2, 0.8)
    xo, sto = oracle.fgmres(A, mg, P.f, tol=1e-10, restart=30, maxit=500)
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-10, restart=30, maxit=500)
    assert st.status == helm.HELM_OK and st.rel_res <= 1e-10
    assert abs(st.iterations - sto["iterations"]) <= 1
    assert rel_l2(to_np(x), xo) <= 1e-8
    # independent residual check with the oracle's operator
    r = P.f - A.apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-10


def test_fgmres_mixed_precision(helm, oracle):
    P = W.config_small(65)
    h = gpu_handle(helm, P, pc="csg", prec="c64")
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, 17, 2, 2, 0.8)
    xo, _ = oracle.fgmres(A, mg, P.f, tol=1e-10, restart=30, maxit=500)
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-10, restart=30, maxit=500)
    assert st.status == helm.HELM_OK
    r = P.f - A.apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-10
    assert rel_l2(to_np(x), xo) <= 1e-7


@pytest.mark.parametrize("gs", ["df", "dcgs2"])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_fgmres_double_float_gram_schmidt(helm, oracle, prec, gs):
    """The double-FP32 Arnoldi on float-pair vectors (CGS + DGKS, or delayed CGS2) reaches the
    same FP64 solution: 1e-8 of the oracle at 1e-10 (FP64 cycle), and the same iteration count
    as FP64 Gram-Schmidt."""
    P = W.config_small(65)
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, 17, 2, 2, 0.8)
    xo, sto = oracle.fgmres(A, mg, P.f, tol=1e-10, restart=30, maxit=500)
    hdf = gpu_handle(helm, P, pc="csg", prec=prec, gs=gs)
    h64 = gpu_handle(helm, P, pc="csg", prec=prec, gs="fp64")
    x, st = helm.krylov_solve(hdf, to_gpu(P.f), tol=1e-10, restart=30, maxit=500)
    x64, st64 = helm.krylov_solve(h64, to_gpu(P.f), tol=1e-10, restart=30, maxit=500)
    assert st.status == helm.HELM_OK
    r = P.f - A.apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-10
    assert abs(st.iterations - st64.iterations) <= 1
    assert rel_l2(to_np(x), xo) <= (1e-8 if prec == "c128" else 1e-7)


@pytest.mark.parametrize("gs", ["df", "dcgs2"])
def test_double_float_gram_schmidt_bench_size(helm, gs):
    """1025 x 1025 well problem (the benchmark workload), complex64 cycle: double-FP32 and FP64
    Gram-Schmidt give the same solution to the accuracy of the solve (rel. residual 1e-8)."""
    P = W.config_2d_well(1025)
    f = to_gpu(P.f)
    out = {}
    for gs in (gs, "fp64"):
        h = gpu_handle(helm, P, pc="csg", prec="c64", gs=gs)
        x, st = helm.krylov_solve(h, f, tol=1e-8, restart=30, maxit=3000)
        assert st.status == helm.HELM_OK and st.rel_res <= 1e-8
        out[gs] = (x, st)
        h.close()
    # restarted GMRES(30) iteration counts at this size can move by a few percent under a
    # change of rounding order
    assert abs(out[gs][1].iterations - out["fp64"][1].iterations) <= 0.1 * out["fp64"][1].iterations
    d = float(torch.linalg.vector_norm(out[gs][0] - out["fp64"][0]) / torch.linalg.vector_norm(out["fp64"][0]))
    assert d <= 1e-6


@pytest.mark.parametrize("restart", [30, 7, 1])
def test_dcgs2_residual_history_matches_cgs(helm, restart):
    """Delayed CGS2 and FP64 CGS + DGKS build the same Krylov method: with an FP64 cycle the
    residual estimates of the first iterations agree to 1e-7 relative, including across
    restarts (restart 7) and with one column per cycle (restart 1, closing step only)."""
    P = W.config_small(65)
    f = to_gpu(P.f)
    hist = {}
    for gs in ("dcgs2", "fp64"):
        h = gpu_handle(helm, P, pc="csg", prec="c128", gs=gs)
        x, st = helm.krylov_solve(h, f, tol=1e-10, restart=restart, maxit=40, history=True,
                                  raise_on_noconv=False)
        hist[gs] = np.array(st.history[: st.iterations])
    k = min(len(hist["dcgs2"]), len(hist["fp64"]), 25)
    assert k >= 10
    a, b = hist["dcgs2"][:k], hist["fp64"][:k]
    assert np.all(np.abs(a - b) <= 1e-7 * b + 1e-13)


@pytest.mark.parametrize("restart,prec", [(30, "c64"), (7, "c64"), (30, "c128")])
def test_dcgs2_solves_after_an_early_stop(helm, restart, prec):
    """Delayed CGS2 queues steps ahead of the host's convergence test (here with a complex64 or a
    complex128 cycle);
    those queued behind a converged step skip their work (a device flag that the rotation kernel
    sets when an estimate meets the current solve's tolerance, cleared at every cycle start).
    Solves of different tolerances in a row on one handle, so with the flag set by the previous
    solve and the replayed step graphs, give bit for bit the iterations and solutions of fresh
    handles."""
    P = W.config_2d_well(129)
    f = to_gpu(P.f)
    tols = (1e-3, 1e-9, 1e-5)

    def solve(h, tol):
        x, st = helm.krylov_solve(h, f, tol=tol, restart=restart, maxit=2000, history=True)
        return x.clone(), st

    h = gpu_handle(helm, P, pc="csg", prec=prec, gs="dcgs2")
    seq = [solve(h, t) for t in tols]
    h.close()
    for t, (x, st) in zip(tols, seq):
        hf = gpu_handle(helm, P, pc="csg", prec=prec, gs="dcgs2")
        xf, stf = solve(hf, t)
        hf.close()
        assert st.status == helm.HELM_OK and st.rel_res <= t
        assert st.iterations == stf.iterations and st.restarts == stf.restarts
        assert np.array_equal(np.array(st.history[: st.iterations]), np.array(stf.history[: stf.iterations]))
        assert torch.equal(x, xf)
    assert seq[0][1].iterations < seq[2][1].iterations < seq[1][1].iterations


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_bicgstab_matches_oracle(helm, oracle, prec):
    P = W.config_small(65)
    h = gpu_handle(helm, P, pc="csg", prec=prec)
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, 17, 2, 2, 0.8)
    xo, sto = oracle.bicgstab(A, mg, P.f, tol=1e-10, maxit=500)
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-10, maxit=500, method="bicgstab")
    assert st.status == helm.HELM_OK
    r = P.f - A.apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 2e-10
    assert rel_l2(to_np(x), xo) <= (1e-8 if prec == "c128" else 1e-7)


@pytest.mark.parametrize("dim,n,pc", [(2, 129, "csl"), (3, 33, "csg"), (2, 65, "qd")])
def test_fgmres_other_configs(helm, oracle, dim, n, pc):
    P = small_problem(dim, n, kh=0.4)
    kw = {}
    if pc == "qd":
        A0, _ = oracle_pair(oracle, P, pc="none")
        kw = dict(re_lambda0=float(np.linalg.eigvals(A0.dense()).real.min()))
    h = gpu_handle(helm, P, pc=pc, prec="c128", smoother="rb" if pc == "qd" else "jacobi",
                   omega=1.0 if pc == "qd" else 0.8, nu=(1, 1) if pc == "qd" else (2, 2), **kw)
    A, M = oracle_pair(oracle, P, pc=pc, **kw)
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-10, restart=30, maxit=2000)
    assert st.status == helm.HELM_OK
    r = P.f - A.apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1.5e-10


def test_solver_status_codes(helm):
    P = W.config_small(33)
    h = gpu_handle(helm, P, pc="csg")
    # zero right-hand side: x = 0 without iterating
    x, st = helm.krylov_solve(h, torch.zeros(P.k2.shape, dtype=torch.complex128, device="cuda"))
    assert st.iterations == 0 and float(x.abs().max()) == 0.0
    # iteration cap
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-14, maxit=3, raise_on_noconv=False)
    assert st.status == helm.HELM_ERR_NOCONV and st.iterations == 3
    with pytest.raises(helm.HelmError) as e:
        helm.krylov_solve(h, to_gpu(P.f), tol=1e-14, maxit=3)
    assert e.value.status == helm.HELM_ERR_NOCONV
    # a NaN injected on the host is reported, not propagated silently
    f = P.f.copy()
    f[5, 5] = np.nan
    with pytest.raises(helm.HelmError) as e:
        helm.krylov_solve(h, to_gpu(f))
    assert e.value.status == helm.HELM_ERR_NONFINITE
    # the handle stays usable
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-8)
    assert st.status == helm.HELM_OK


def test_residual_history_monotone(helm):
    P = W.config_small(65)
    h = gpu_handle(helm, P, pc="csg", prec="c128")
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-10, restart=30, history=True)
    hist = np.array(st.history[:30])
    assert np.all(np.diff(hist) <= 1e-12)


# ---------------------------------------------------------------------------- adjoint

def test_adjoint_matches_dense(helm, oracle):
    P = small_problem(2, 17, kh=0.5)
    h = gpu_handle(helm, P, pc="csg", prec="c128")
    A, _ = oracle_pair(oracle, P)
    g = W.random_field(P.k2.shape, 61)
    lam, st = helm.helm_solve_adjoint(h, to_gpu(g), tol=1e-12)
    ref = np.zeros_like(g)
    ref[1:-1, 1:-1] = np.linalg.solve(A.dense().T, g[1:-1, 1:-1].ravel()).reshape(15, 15)
    assert rel_l2(to_np(lam), ref) <= 1e-9
    u = W.random_field(P.k2.shape, 62)
    grad = to_np(helm.helm_grad_k2(h, to_gpu(ref), to_gpu(u)))
    exp = np.zeros(P.k2.shape)
    exp[1:-1, 1:-1] = np.real(ref * u)[1:-1, 1:-1]
    assert np.abs(grad - exp).max() <= 1e-14 * np.abs(exp).max()


def test_autograd_gradient_central_differences(helm):
    """L = |sum g u|^2, u = A(k^2)^{-1} f; torch.autograd through HelmholtzSolve against central
    differences (step 1e-6) at seeded points, forward pairs solved to 1e-13."""
    n = 33
    P = small_problem(2, n, kh=0.5)
    g = to_gpu(W.gaussian_source(2, n, 0.1, 77).real)

    def factory(k2):
        P2 = W.Problem("t", 2, n, k2.cpu().numpy(), P.f, coarsest_n=17)
        return gpu_handle(helm, P2, pc="csg", prec="c128")

    k2 = to_gpu(P.k2).requires_grad_(True)
    f = to_gpu(P.f)
    u = helm.HelmholtzSolve.apply(k2, f, factory, 1e-13, 30, 2000)
    L = (g.to(u.dtype) * u).sum().abs() ** 2
    L.backward()
    grad = to_np(k2.grad)
    rng = np.random.default_rng(5)
    pts = rng.integers(1, n - 1, size=(8, 2))
    gmax = np.abs(grad).max()
    for (j, i) in pts:
        vals = []
        for sgn in (1, -1):
            kk = P.k2.copy()
            kk[j, i] += sgn * 1e-6
            hh = factory(torch.from_numpy(kk))
            uu, _ = helm.krylov_solve(hh, f, tol=1e-13, maxit=2000)
            vals.append(float(((g.to(uu.dtype) * uu).sum().abs() ** 2).item()))
        fd = (vals[0] - vals[1]) / 2e-6
        # normwise: the difference quotient carries ~tol * L / step of solver noise
        assert abs(fd - grad[j, i]) <= 1e-5 * gmax
        if abs(grad[j, i]) > 0.1 * gmax:
            assert abs(fd - grad[j, i]) <= 1e-4 * abs(grad[j, i])
