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
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", gs="df", coarsest_n=17)
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
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-14, restart=30, maxit=4, raise_on_noconv=False)
    assert all(st.status == helm.HELM_ERR_NOCONV and st.iterations == 4 for st in stats)


def test_autotuned_batch_matches_single_solves_with_the_same_tuning(helm, tmp_path):
    probs = W.config_batch(count=5, seed=13, sizes=(129, 257))
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", gs="df", coarsest_n=17)
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


# ---------------------------------------------------------------------------- lockstep engine

def lockstep_batch(helm, count, seed, sizes, engine="auto"):
    probs = W.config_batch(count=count, seed=seed, sizes=sizes)
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", gs="dcgs2", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    helm.helm_batch_set_engine(b, engine)
    return probs, b


def test_lockstep_batch_matches_single_solves(helm, oracle):
    """The lockstep engine (every phase of an FGMRES step one launch over all problems) gives
    each problem the result of krylov_solve on a handle with the tuning the engine installed:
    the same iteration count and the same solution bit for bit; the residuals are checked with
    the oracle's operator."""
    probs, b = lockstep_batch(helm, 6, 21, (129, 257, 513))
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-9, restart=30, maxit=3000)
    torch.cuda.synchronize()
    assert helm.helm_batch_get_engine(b) == "lockstep"
    assert len({P.n for P in probs}) >= 2
    for i, (P, r, x, st) in enumerate(zip(probs, rhs, xs, stats)):
        assert st.status == helm.HELM_OK and st.rel_res <= 1e-9
        hb = helm.batch_handle(b, i)
        h = gpu_handle(helm, P, pc="csg", prec="c64", gs="dcgs2")
        helm.helm_set_tuning(h, helm.helm_get_tuning(hb))
        x1, st1 = helm.krylov_solve(h, r, tol=1e-9, restart=30, maxit=3000)
        assert st1.iterations == st.iterations, (P.n, st1.iterations, st.iterations)
        assert torch.equal(x, x1), float(torch.linalg.vector_norm(x - x1) / torch.linalg.vector_norm(x1))
        A, _ = oracle_pair(oracle, P)
        res = P.f - A.apply(to_np(x))
        assert np.linalg.norm(res) / np.linalg.norm(P.f) <= 1.5e-9


def test_lockstep_and_streams_engines_agree(helm):
    """The same batch solved by both engines: same iterations, same solutions."""
    out = {}
    for engine in ("lockstep", "streams"):
        probs, b = lockstep_batch(helm, 5, 22, (129, 257), engine=engine)
        if engine == "streams":
            # the streams engine runs each handle's own tuning: give it the lockstep's
            for i in range(len(probs)):
                helm.helm_set_tuning(helm.batch_handle(b, i), out["lockstep"][2][i])
        rhs = [to_gpu(P.f) for P in probs]
        xs = [torch.zeros_like(r) for r in rhs]
        stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-9, restart=30, maxit=3000)
        torch.cuda.synchronize()
        assert helm.helm_batch_get_engine(b) == engine
        out[engine] = (xs, stats, [helm.helm_get_tuning(helm.batch_handle(b, i)) for i in range(len(probs))])
    for xa, xb_, sa, sb in zip(out["lockstep"][0], out["streams"][0], out["lockstep"][1], out["streams"][1]):
        assert sa.iterations == sb.iterations
        assert torch.equal(xa, xb_)


def test_lockstep_status_and_restarts(helm):
    """Per-problem caps and statuses in lockstep: an iteration cap below one restart cycle, and
    a cap that spans several restarts (restart 7)."""
    probs, b = lockstep_batch(helm, 4, 23, (129, 257))
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-14, restart=30, maxit=4, raise_on_noconv=False)
    assert helm.helm_batch_get_engine(b) == "lockstep"
    assert all(st.status == helm.HELM_ERR_NOCONV and st.iterations == 4 for st in stats)
    for x in xs:
        x.zero_()
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-9, restart=7, maxit=3000)
    for i, (P, r, x, st) in enumerate(zip(probs, rhs, xs, stats)):
        assert st.status == helm.HELM_OK and st.restarts >= 2
        h = gpu_handle(helm, P, pc="csg", prec="c64", gs="dcgs2")
        helm.helm_set_tuning(h, helm.helm_get_tuning(helm.batch_handle(b, i)))
        x1, st1 = helm.krylov_solve(h, r, tol=1e-9, restart=7, maxit=3000)
        assert st1.iterations == st.iterations and torch.equal(x, x1)


def test_lockstep_solves_after_an_early_stop(helm):
    """The batched rotation takes a converged problem out of the steps already queued behind it
    (its flag cleared on the device, tested against the current solve's tolerance): batch solves
    of different tolerances in a row give each problem what a single solve gives, bit for bit."""
    probs, b = lockstep_batch(helm, 4, 25, (129, 257))
    rhs = [to_gpu(P.f) for P in probs]
    for tol in (1e-4, 1e-9, 1e-6):
        xs = [torch.zeros_like(r) for r in rhs]
        stats = helm.helm_solve_batch(b, rhs, xs, tol=tol, restart=30, maxit=3000)
        assert helm.helm_batch_get_engine(b) == "lockstep"
        for i, (P, r, x, st) in enumerate(zip(probs, rhs, xs, stats)):
            assert st.status == helm.HELM_OK and st.rel_res <= tol
            h = gpu_handle(helm, P, pc="csg", prec="c64", gs="dcgs2")
            helm.helm_set_tuning(h, helm.helm_get_tuning(helm.batch_handle(b, i)))
            x1, st1 = helm.krylov_solve(h, r, tol=tol, restart=30, maxit=3000)
            h.close()
            assert st1.iterations == st.iterations and torch.equal(x, x1)


def test_lockstep_rejects_other_configurations(helm):
    probs = W.config_batch(count=2, seed=24, sizes=(129,))
    mg = helm.MGParams(kind="csg", theta_a=probs[0].theta_a, prec="c64", gs="df", coarsest_n=17)
    specs = [dict(dim=2, n=P.n, k2=torch.from_numpy(P.k2), theta=P.theta) for P in probs]
    b = helm.helm_create_batch(specs, mg=mg)
    helm.helm_batch_set_engine(b, "lockstep")
    rhs = [to_gpu(P.f) for P in probs]
    xs = [torch.zeros_like(r) for r in rhs]
    with pytest.raises(helm.HelmError) as e:
        helm.helm_solve_batch(b, rhs, xs, tol=1e-9)
    assert e.value.status == helm.HELM_ERR_ARG and "lockstep" in str(e.value)
    helm.helm_batch_set_engine(b, "auto")
    stats = helm.helm_solve_batch(b, rhs, xs, tol=1e-9)
    assert helm.helm_batch_get_engine(b) == "streams" and all(st.status == helm.HELM_OK for st in stats)
