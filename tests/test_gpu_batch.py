"""Batched solves (many energies and grid sizes at once) against one-at-a-time solves and the
oracle's residual."""
import math

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


def test_batch_matches_single_solves(helm, oracle):
    probs = W.config_batch(count=7, seed=11, sizes=(33, 65, 129))
    mg = helm.MGParams(kind="csg", prec="c64", gs="df", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-9, restart=30, maxit=2000)
    torch.cuda.synchronize()
    for P, r, x, st in zip(probs, rhs, xs, stats):
        assert st.status == helm.HELM_OK
        h = gpu_handle(helm, P, pc="csg", prec="c64", gs="df")
        x1, st1 = helm.krylov_solve(h, r, tol=1e-9, restart=30, maxit=2000)
        assert st1.iterations == st.iterations
        assert float(torch.linalg.vector_norm(x - x1)) <= 1e-12 * float(torch.linalg.vector_norm(x1))
        A, _ = oracle_pair(oracle, P)
        res = P.f - A.apply(to_np(x))
        assert np.linalg.norm(res) / np.linalg.norm(P.f) <= 1.5e-9


def test_batch_reports_per_problem_status(helm):
    probs = W.config_batch(count=3, seed=12, sizes=(33, 65))
    mg = helm.MGParams(kind="csg", prec="c64", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-14, restart=30, maxit=4, raise_on_noconv=False)
    assert all(st.status == helm.HELM_ERR_NOCONV and st.iterations == 4 for st in stats)


def test_autotuned_batch_matches_single_solves_with_the_same_tuning(helm, tmp_path):
    probs = W.config_batch(count=5, seed=13, sizes=(129, 257))
    mg = helm.MGParams(kind="csg", prec="c64", gs="df", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    chosen = helm.helm_autotune_batch(b, "c64", reps=3, cache=str(tmp_path / "t.json"))
    assert len(chosen) == len({P.n for P in probs})
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-9, restart=30, maxit=2000)
    torch.cuda.synchronize()
    for i, (P, r, x, st) in enumerate(zip(probs, rhs, xs, stats)):
        assert st.status == helm.HELM_OK
        hb = helm.batch_handle(b, i)
        assert helm.helm_get_tuning(hb) == chosen[helm.tuning_key(hb, "c64")]
        h = gpu_handle(helm, P, pc="csg", prec="c64", gs="df")
        helm.helm_set_tuning(h, helm.helm_get_tuning(hb))
        x1, st1 = helm.krylov_solve(h, r, tol=1e-9, restart=30, maxit=2000)
        assert st1.iterations == st.iterations
        assert float(torch.linalg.vector_norm(x - x1)) <= 1e-12 * float(torch.linalg.vector_norm(x1))
