"""Full-size workloads (the grids the benchmark and the problem configurations name), solved the
way the benchmark solves them (complex64 cycle with the autotuned kernels, double-FP32 delayed
CGS2 Arnoldi).  Each solution is checked with the oracle's own operator (the Section 3.2
stencil on the ECS grid, written independently in C): the relative residual ||f - A x|| / ||f||
the oracle computes must meet the tolerance the solve was asked for, up to rounding."""
import numpy as np
import pytest

from helpers import gpu_handle, oracle_pair, to_gpu, to_np
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


def oracle_rel_residual(oracle, P, x):
    A, _ = oracle_pair(oracle, P)
    r = P.f - A.apply(x)
    return float(np.linalg.norm(r) / np.linalg.norm(P.f))


def test_2d_1025_well_benchmark_solve(helm, oracle, tmp_path):
    P = W.config_2d_well(1025)
    h = gpu_handle(helm, P, pc="csg", prec="c64", gs="dcgs2")
    helm.helm_autotune(h, "c64", reps=5, cache=str(tmp_path / "t.json"))
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-8, restart=30, maxit=3000)
    assert st.status == helm.HELM_OK and st.rel_res <= 1e-8
    assert oracle_rel_residual(oracle, P, to_np(x)) <= 1.0001e-8


def test_3d_257_well_solve(helm, oracle, tmp_path):
    """255^3 = 16.6 M unknowns, FGMRES(20), 7-point stencil, ECS on all faces."""
    P = W.config_3d_well(257)
    h = gpu_handle(helm, P, pc="csg", prec="c64", gs="dcgs2")
    helm.helm_autotune(h, "c64", reps=3, cache=str(tmp_path / "t.json"))
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-8, restart=20, maxit=4000)
    assert st.status == helm.HELM_OK and st.rel_res <= 1e-8
    assert oracle_rel_residual(oracle, P, to_np(x)) <= 1.0001e-8


def test_batch_of_64_mixed_sizes(helm, oracle, tmp_path):
    probs = W.config_batch(64)
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", gs="dcgs2", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    helm.helm_autotune_batch(b, "c64", reps=3, cache=str(tmp_path / "t.json"))
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-8, restart=30, maxit=5000)
    torch.cuda.synchronize()
    for P, x, st in zip(probs, xs, stats):
        assert st.status == helm.HELM_OK and st.rel_res <= 1e-8
        assert oracle_rel_residual(oracle, P, to_np(x)) <= 1.0001e-8, P.name
