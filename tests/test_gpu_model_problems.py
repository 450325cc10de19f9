"""CUDA path against the CPU oracle, element by element, on the geometry of the paper's model
problems (Section 6, Tables 1-4), which the other parity tests do not cover:

* MP1: ECS layers on all four sides of a shifted square ([-1/2, 1/2]^2 interior, 64 layer
  cells per side, 385 x 385 nodes) and a point source;
* MP2 / MP3: layers on the north and east sides only (Dirichlet at x = 0 and y = 0) of the
  square [0, 50] plus a 12.5-wide layer (641 x 641 nodes), with the potentials
  nu (exp(-x^2) + exp(-y^2)) and 1/x + 1/y and the source exp(-(x^2 + y^2)).

Checked: the operator apply A and every preconditioning operator M (1e-14, relative l2 on
random input), one cycle of Algorithm 1 with each table's cycle and smoother in FP64 (1e-12),
the Bi-CGSTAB iterate after a fixed number of iterations (the same method step by step,
1e-8), and full Bi-CGSTAB solutions on reduced grids of the same geometry (1e-8 at a relative
residual of 1e-11)."""
import json
import math
import os

import numpy as np
import pytest

from helpers import gpu_handle, oracle_pair, rel_l2, to_gpu, to_np
from paper_1012_4307_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))

FULL = {
    "mp1": lambda: W.paper_mp1(k=160.0),
    "mp2": lambda: W.paper_mp2(k=4.0, nu=7.0),
    "mp3": lambda: W.paper_mp3(k=2.0),
}
TABLE_OF = {"mp1": "T1", "mp2": "T2", "mp3": "T3"}


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_4307_gb300 import helm as H
    H.load()
    return H


@pytest.fixture(scope="module")
def problems():
    return {k: f() for k, f in FULL.items()}


def table_kw(table, pc):
    """Preconditioner and cycle parameters of a table's row (Tables 1-4)."""
    c = GOLDEN[table][pc]
    kw = dict(pc=pc, smoother=c["smoother"], nu=(1, 1), omega=c["omega"], gamma=(1, c["gamma_c"]))
    okw = dict(pc=pc)
    if "beta" in c:
        kw["beta"] = okw["beta"] = tuple(c["beta"])
    if "theta_a_pi_over" in c:
        kw["theta_a"] = okw["theta_a"] = math.pi / c["theta_a_pi_over"]
    if "re_lambda0" in c:
        kw["re_lambda0"] = okw["re_lambda0"] = c["re_lambda0"]
    return kw, okw


def test_geometry_is_the_papers(problems):
    """The builders give the printed grids: MP1 256 + 2 x 64 cells per axis with layers on both
    sides, MP2/MP3 512 + 128 cells with one layer (north/east), and a point source for MP1."""
    p1, p2 = problems["mp1"], problems["mp2"]
    assert p1.n == 385 and p2.n == 641
    assert p1.layers == (-0.5, 0.5) and p1.lo == -0.75 and p1.hi == 0.75
    assert p2.lo == 0.0 and p2.layers[0] < p2.lo and p2.layers[1] == 50.0 and p2.hi == 62.5
    assert np.count_nonzero(p1.f) == 1


@pytest.mark.parametrize("mp", ["mp1", "mp2", "mp3"])
@pytest.mark.parametrize("pc", ["csl", "csg", "qd"])
def test_model_problem_apply(helm, oracle, problems, mp, pc):
    P = problems[mp]
    kw, okw = table_kw(TABLE_OF[mp], pc)
    h = gpu_handle(helm, P, prec="c128", **kw)
    A, M = oracle_pair(oracle, P, **okw)
    x = W.random_field(P.k2.shape, 500 + len(mp))
    for which, op in (("A", A), ("M", M)):
        y = helm.helm_apply(h, to_gpu(x), which=which)
        assert rel_l2(to_np(y), op.apply(x)) <= 1e-14, (mp, pc, which)
    h.close()


@pytest.mark.parametrize("mp", ["mp1", "mp2", "mp3"])
@pytest.mark.parametrize("pc", ["csl", "csg", "qd"])
def test_model_problem_cycle(helm, oracle, problems, mp, pc):
    """One cycle of the table's F_1^gc(1,1) (CSL, CSG) or V(1,1) red-black (QD) in FP64, from
    zero on the model problem's own right-hand side and from a random guess."""
    P = problems[mp]
    table = TABLE_OF[mp]
    kw, okw = table_kw(table, pc)
    h = gpu_handle(helm, P, prec="c128", **kw)
    A, M = oracle_pair(oracle, P, **okw)
    mg = oracle.MG(M, P.coarsest_n, 1, 1, kw["omega"], kw["smoother"])
    assert h.levels == [mg.level_shape(l) for l in range(mg.nlev)]
    gam = kw["gamma"]
    b = P.f
    x = helm.mg_vcycle(h, to_gpu(b))
    assert rel_l2(to_np(x), mg.cycle(b, None, *gam)) <= 1e-12
    u0 = W.random_field(P.k2.shape, 600)
    b2 = W.random_field(P.k2.shape, 601)
    x = helm.mg_vcycle(h, to_gpu(b2), to_gpu(u0))
    assert rel_l2(to_np(x), mg.cycle(b2, u0, *gam)) <= 1e-12
    h.close()


@pytest.mark.parametrize("mp,pc,iters", [("mp1", "csg", 12), ("mp2", "csl", 8), ("mp3", "qd", 8)])
def test_model_problem_bicgstab_iterate(helm, oracle, problems, mp, pc, iters):
    """Bi-CGSTAB (two cycles per iteration, Section 5) with the table's preconditioner: after
    the same number of iterations the GPU iterate equals the oracle's to 1e-8 (the two run the
    same method in FP64; only the order of rounding differs)."""
    P = problems[mp]
    kw, okw = table_kw(TABLE_OF[mp], pc)
    h = gpu_handle(helm, P, prec="c128", **kw)
    A, M = oracle_pair(oracle, P, **okw)
    mg = oracle.MG(M, P.coarsest_n, 1, 1, kw["omega"], kw["smoother"])
    xo, sto = oracle.bicgstab(A, mg, P.f, tol=1e-14, maxit=iters, gamma_f=1, gamma_c=kw["gamma"][1])
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-14, maxit=iters, method="bicgstab", raise_on_noconv=False)
    assert st.iterations == sto["iterations"] == iters
    assert rel_l2(to_np(x), xo) <= 1e-8
    h.close()


REDUCED = {
    # the printed geometry at a quarter of the width, same mesh width (h = 50/512)
    "mp2": lambda: W.paper_mp2(k=4.0, nu=7.0, size=12.5, interior_cells=128, layer_cells=32),
    "mp3": lambda: W.paper_mp3(k=2.0, size=12.5, interior_cells=128, layer_cells=32),
    # MP1 with k h as printed (160 / 256) on 64 + 2 x 16 cells per axis
    "mp1": lambda: W.paper_mp1(k=40.0, interior_cells=64, layer_cells=16),
}


@pytest.mark.parametrize("mp", ["mp1", "mp2", "mp3"])
def test_model_problem_solution(helm, oracle, mp):
    """Full Bi-CGSTAB solves with the table's CSG row (FP64) on a reduced grid of the same
    geometry: both reach a relative residual of 1e-11 and their solutions agree to 1e-8."""
    P = REDUCED[mp]()
    kw, okw = table_kw(TABLE_OF[mp], "csg")
    h = gpu_handle(helm, P, prec="c128", **kw)
    A, M = oracle_pair(oracle, P, **okw)
    mg = oracle.MG(M, P.coarsest_n, 1, 1, kw["omega"], kw["smoother"])
    xo, sto = oracle.bicgstab(A, mg, P.f, tol=1e-11, maxit=3000, gamma_f=1, gamma_c=kw["gamma"][1])
    x, st = helm.krylov_solve(h, to_gpu(P.f), tol=1e-11, maxit=3000, method="bicgstab")
    assert st.status == helm.HELM_OK and sto["status"] == 0
    r = P.f - A.apply(to_np(x))
    assert np.linalg.norm(r) / np.linalg.norm(P.f) <= 1e-10
    assert rel_l2(to_np(x), xo) <= 1e-8
    h.close()
