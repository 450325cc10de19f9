"""Cycle tuning (kernel choices) and the autotuner: every choice of tail depth and tile shape
is the same cycle of Algorithm 1 (checked against the oracle's cycle, Section 4.2, on the
preconditioner call of Section 5), and the autotuned solve reaches the same solution."""
import json

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


def problem(n):
    return W.Problem("t", 2, n, W.k2_well_growth(2, n, kh_max=0.5), W.gaussian_source(2, n, 0.1, 0), coarsest_n=17)


@pytest.mark.parametrize("n", [257, 1025])
def test_every_tuning_is_the_same_cycle(helm, oracle, n):
    P = problem(n)
    h = gpu_handle(helm, P, pc="csg", prec="c64")
    A, M = oracle_pair(oracle, P)
    mg = oracle.MG(M, P.coarsest_n, 2, 2, 0.8, "jacobi")
    v = W.random_field(P.k2.shape, 41)
    ref = mg.cycle(v)
    vg = to_gpu(v)
    nlev = len(h.levels)
    choices = [dict(tail_levels=t, level_tile=[tile] * nlev) for t in (0, 2, 3)
               for tile in ("none", "32x8", "16x16", "16x8", "64x4", "wave", "8x8")]
    mixed = ["64x4", "wave", "16x8", "8x8", "16x16", "32x8", "none"]
    choices.append(dict(tail_levels=-1, level_tile=[mixed[l % len(mixed)] for l in range(nlev)]))
    # thread-block-cluster tails over the coarsest 2 .. 5 levels, 8 or 16 blocks, 1 or 3 halo rows
    for cl in (2, 3, 4, 5):
        for nc in (8, 16):
            for halo in (1, 3):
                choices.append(dict(tail_levels=0, level_tile=["16x8"] * nlev, cluster_levels=cl, cluster_ctas=nc,
                                    cluster_halo=halo))
    for c in choices:
        c.setdefault("cluster_levels", 0)
        c.setdefault("cluster_ctas", 16)
        c.setdefault("cluster_halo", 3)
        helm.helm_set_tuning(h, c)
        got = helm.helm_get_tuning(h)
        assert got == c
        z = to_np(helm.mg_precondition(h, vg))
        assert rel_l2(z, ref) <= 2e-5, c


def test_autotune_installs_a_choice_and_solves_the_same(helm, tmp_path):
    P = W.config_2d_well(513)
    f = to_gpu(P.f)
    h = gpu_handle(helm, P, pc="csg", prec="c64", gs="df")
    x0, st0 = helm.krylov_solve(h, f, tol=1e-8, restart=30, maxit=3000)
    cache = str(tmp_path / "tuning.json")
    tuning, ms = helm.helm_autotune(h, "c64", reps=5, cache=cache)
    assert ms > 0 and helm.helm_get_tuning(h) == tuning
    x1, st1 = helm.krylov_solve(h, f, tol=1e-8, restart=30, maxit=3000)
    assert st1.status == helm.HELM_OK and st1.rel_res <= 1e-8
    # same problem to the solve's accuracy; iteration counts may move under FP32 rounding order
    d = float(torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0))
    assert d <= 1e-6
    assert abs(st1.iterations - st0.iterations) <= 0.1 * st0.iterations + 2
    # the cache returns the stored choice without timing
    table = json.load(open(cache))
    assert helm.tuning_key(h, "c64") in table
    h2 = gpu_handle(helm, P, pc="csg", prec="c64", gs="df")
    t2, ms2 = helm.helm_autotune(h2, "c64", cache=cache)
    assert t2 == tuning and ms2 == ms and helm.helm_get_tuning(h2) == tuning


def test_set_tuning_rejects_bad_values(helm):
    P = problem(65)
    h = gpu_handle(helm, P, pc="csg", prec="c64")
    with pytest.raises(helm.HelmError):
        helm.helm_set_tuning(h, dict(tail_levels=1))
    with pytest.raises(helm.HelmError):
        helm.helm_set_tuning(h, dict(tail_levels=-2))
    with pytest.raises(helm.HelmError):
        helm.helm_set_tuning(h, dict(cluster_levels=1))
    with pytest.raises(helm.HelmError):
        helm.helm_set_tuning(h, dict(cluster_levels=2, cluster_ctas=4))
    with pytest.raises(helm.HelmError):
        helm.helm_set_tuning(h, dict(cluster_levels=2, cluster_halo=2))


@pytest.mark.parametrize("smoother,nu,gamma", [("rb", (1, 1), (1, 2)), ("jacobi", (1, 2), (2, 2)), ("jacobi", (0, 1), (1, 1))])
def test_cluster_tail_general_cycles(helm, oracle, smoother, nu, gamma):
    """The cluster tail follows Algorithm 1 for red-black smoothing, W/F cycles and uneven
    sweep counts too (checked against the oracle's cycle, complex64 tolerance)."""
    P = problem(129)
    h = gpu_handle(helm, P, pc="csl", prec="c64", smoother=smoother, nu=nu, gamma=gamma, omega=0.8)
    A, M = oracle_pair(oracle, P, pc="csl")
    mg = oracle.MG(M, P.coarsest_n, nu[0], nu[1], 0.8, smoother)
    v = W.random_field(P.k2.shape, 43)
    ref = mg.cycle(v, None, *gamma)
    nlev = len(h.levels)
    for cl in (2, 3, nlev):
        helm.helm_set_tuning(h, dict(tail_levels=0, level_tile=["none"] * nlev, cluster_levels=cl, cluster_ctas=8))
        z = to_np(helm.mg_precondition(h, to_gpu(v)))
        assert rel_l2(z, ref) <= 2e-5, cl


def kernel_names(fn):
    """Names of the CUDA kernels fn launches (torch's profiler); None when it records none."""
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    names = {e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA}
    return names or None


@pytest.mark.parametrize("n", [129, 257, 1025])
@pytest.mark.parametrize("nu", [(2, 2), (1, 2), (2, 1), (0, 1), (1, 0)])
def test_deep_halo_cluster_tail_equals_one_row_tail(helm, n, nu):
    """With three halo rows each block recomputes the rows next to its slab from the same
    operands with the same operations as their owner, so the cycle equals the one-row cluster
    tail's bit for bit, for every tail depth and cluster size that fits."""
    P = problem(n)
    h = gpu_handle(helm, P, pc="csg", prec="c64", nu=nu)
    nlev = len(h.levels)
    v = to_gpu(W.random_field(P.k2.shape, 44))
    ran_deep = False
    for cl in (2, 3, 4, 5):
        for nc in (8, 16):
            outs = []
            for halo in (1, 3):
                helm.helm_set_tuning(h, dict(tail_levels=0, level_tile=["16x8"] * nlev, cluster_levels=cl,
                                             cluster_ctas=nc, cluster_halo=halo))
                outs.append(helm.mg_precondition(h, v))
                if halo == 3 and not ran_deep:
                    names = kernel_names(lambda: helm.mg_precondition(h, v))
                    ran_deep = names is None or any("k_mg_chalo" in s for s in names)
            assert torch.equal(outs[0], outs[1]), (cl, nc)
    assert ran_deep


@pytest.mark.parametrize("nx,ny", [(257, 129), (129, 257)])
def test_deep_halo_cluster_tail_on_nonsquare_grids(helm, oracle, nx, ny):
    """Non-square grids (each block owns a slab of rows of every level, the columns whole): the
    three-row cluster tail equals the one-row tail bit for bit, and both follow the oracle's
    cycle to complex64 accuracy, for every tail depth and cluster size that fits."""
    k2 = np.ascontiguousarray(W.k2_well_growth(2, max(nx, ny), kh_max=0.5)[:ny, :nx])
    P = W.Problem("ns", 2, [nx, ny], k2, np.zeros((ny, nx), complex), coarsest_n=17)
    h = gpu_handle(helm, P, pc="csg", prec="c64")
    A, M = oracle_pair(oracle, P)
    v = W.random_field((ny, nx), 45)
    ref = oracle.MG(M, P.coarsest_n, 2, 2, 0.8, "jacobi").cycle(v)
    vg = to_gpu(v)
    nlev = len(h.levels)
    for cl in range(2, nlev + 1):
        for nc in (8, 16):
            outs = []
            for halo in (1, 3):
                helm.helm_set_tuning(h, dict(tail_levels=0, level_tile=["16x8"] * nlev, cluster_levels=cl,
                                             cluster_ctas=nc, cluster_halo=halo))
                z = helm.mg_precondition(h, vg)
                assert rel_l2(to_np(z), ref) <= 2e-5, (cl, nc, halo)
                outs.append(z)
            assert torch.equal(outs[0], outs[1]), (cl, nc)
