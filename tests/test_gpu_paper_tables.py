"""The paper's model problems MP1-MP3 (Section 6) with the preconditioners and cycles of
Tables 1-4: Bi-CGSTAB with one cycle per preconditioner call (FP64 cycle and vectors) to a
relative residual of 1e-6, and the stand-alone multigrid convergence of each preconditioner,
against the printed numbers (tests/golden/paper_tables.json): every solve converges, the
multigrid cycle counts equal the printed ones, factors and Bi-CGSTAB iteration counts come
close, and the paper's comparative findings hold (QD needs more Krylov iterations than CSL
and CSG, and its multigrid converges faster than theirs)."""
import json
import math
import os

import pytest

from helpers import gpu_handle, to_gpu
from paper_1012_4307_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
BUILDERS = {"mp1": W.paper_mp1, "mp2": W.paper_mp2, "mp3": W.paper_mp3}


@pytest.fixture(scope="module")
def helm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_4307_gb300 import helm as H
    H.load()
    return H


def run_table(helm, table):
    spec = GOLDEN[table]
    P = BUILDERS[spec["problem"]](**spec["args"])
    f = to_gpu(P.f)
    out = {}
    for pc in ("csl", "csg", "qd"):
        c = spec[pc]
        kw = dict(pc=pc, prec="c128", smoother=c["smoother"], nu=(1, 1), omega=c["omega"], gamma=(1, c["gamma_c"]))
        if "beta" in c:
            kw["beta"] = tuple(c["beta"])
        if "theta_a_pi_over" in c:
            kw["theta_a"] = math.pi / c["theta_a_pi_over"]
        if "re_lambda0" in c:
            kw["re_lambda0"] = c["re_lambda0"]
        h = gpu_handle(helm, P, **kw)
        x, st = helm.krylov_solve(h, f, tol=P.tol, method="bicgstab", maxit=5000)
        _, cycles, factor = helm.helm_mg_conv(h, f, tol=1e-6, maxcyc=500)
        out[pc] = dict(iterations=st.iterations, rel_res=st.rel_res, status=st.status, mg_conv=factor,
                       mg_cycles=cycles, paper=dict(iterations=c["iterations"], mg_conv=c["mg_conv"],
                                                    mg_cycles=c["mg_cycles"]))
        h.close()
    return out


@pytest.mark.parametrize("table", ["T1", "T2", "T3", "T4"])
def test_paper_model_problem(helm, table):
    out = run_table(helm, table)
    print("\n%s %s" % (table, json.dumps(out)))
    for pc, r in out.items():
        assert r["status"] == helm.HELM_OK and r["rel_res"] <= 1e-6, (pc, r)
        # against the printed numbers: the stand-alone multigrid needs exactly the printed cycle
        # count, its factor comes within 0.06, and Bi-CGSTAB within 15% of the printed iterations
        p = r["paper"]
        assert r["mg_cycles"] == p["mg_cycles"], (pc, r)
        assert abs(r["mg_conv"] - p["mg_conv"]) <= 0.06, (pc, r)
        assert abs(r["iterations"] - p["iterations"]) <= 0.15 * p["iterations"], (pc, r)
    assert out["qd"]["iterations"] > max(out["csl"]["iterations"], out["csg"]["iterations"])
    assert out["qd"]["mg_conv"] < min(out["csl"]["mg_conv"], out["csg"]["mg_conv"])


def test_preconditioner_solution_as_starting_guess(helm):
    """Experiment 1's remark (Section 6): with the QD preconditioner, the paper started
    Bi-CGSTAB from the preconditioner's solution, computed by stand-alone multigrid to 1e-2, and
    saw 50 fewer iterations.  QD in its table form is (1-i) I + Z / |Re lambda0|, so its solution
    approximates |Re lambda0| Z^-1 f: started as it is, Bi-CGSTAB needs more iterations than from
    zero (the start's residual is about 2e4 ||f||); divided by |Re lambda0| it is a start with a
    residual of about 0.3 ||f||.  All three solves must converge; the counts are printed (the
    oracle's: 172 from zero, 247 and 165 from the two starts; on GB300: 167, 249 and 172)."""
    spec = GOLDEN["T1"]
    c = spec["qd"]
    P = BUILDERS[spec["problem"]](**spec["args"])
    f = to_gpu(P.f)
    h = gpu_handle(helm, P, pc="qd", prec="c128", smoother=c["smoother"], nu=(1, 1), omega=c["omega"],
                   gamma=(1, c["gamma_c"]), re_lambda0=c["re_lambda0"])
    _, st0 = helm.krylov_solve(h, f, tol=P.tol, method="bicgstab", maxit=5000)
    x0, cycles, _ = helm.helm_mg_conv(h, f, tol=1e-2, maxcyc=100)
    _, st1 = helm.krylov_solve(h, f, x0.clone(), tol=P.tol, method="bicgstab", maxit=5000)
    _, st2 = helm.krylov_solve(h, f, x0 / abs(c["re_lambda0"]), tol=P.tol, method="bicgstab", maxit=5000)
    h.close()
    print("\nfrom zero: %d iterations; from the 1e-2 preconditioner solution (%d cycles): %d; "
          "the same divided by |Re lambda0|: %d" % (st0.iterations, cycles, st1.iterations, st2.iterations))
    for st in (st0, st1, st2):
        assert st.status == helm.HELM_OK and st.rel_res <= P.tol
    # the scaled start is the better one (the unscaled start's residual is about 2e4 ||f||),
    # and the counts from zero and from the scaled start stay within the 15% that the table
    # tests allow of the oracle's 172 and 165
    assert st2.iterations < st1.iterations
    assert abs(st0.iterations - 172) <= 0.15 * 172
    assert abs(st2.iterations - 165) <= 0.15 * 165


@pytest.mark.parametrize("table", ["T1", "T2", "T3", "T4"])
def test_qd_with_computed_lambda0(helm, table):
    """QD with Re(lambda0) from the one-dimensional counterpart (helm_qd_lambda0, Section 6's
    closing remark) instead of the printed value: the stand-alone multigrid still needs the
    printed number of cycles and Bi-CGSTAB still converges, within 25% of the printed count."""
    spec = GOLDEN[table]
    c = spec["qd"]
    P = BUILDERS[spec["problem"]](**spec["args"])
    lam0 = helm.helm_qd_lambda0(2, [P.n, P.n], P.extra["k2_axis"], theta=P.theta, r0_lo=[P.layers[0]] * 2,
                                r0_hi=[P.layers[1]] * 2, lo=[P.lo] * 2, hi=[P.hi] * 2)
    f = to_gpu(P.f)
    h = gpu_handle(helm, P, pc="qd", prec="c128", smoother=c["smoother"], nu=(1, 1), omega=c["omega"],
                   gamma=(1, c["gamma_c"]), re_lambda0=lam0)
    _, cycles, factor = helm.helm_mg_conv(h, f, tol=1e-6, maxcyc=500)
    _, st = helm.krylov_solve(h, f, tol=P.tol, method="bicgstab", maxit=5000)
    h.close()
    print("\n%s QD: Re lambda0 %.6g (printed %.6g), mg cycles %d (printed %d), factor %.3f, Bi-CGSTAB %d (printed %d)"
          % (table, lam0, c["re_lambda0"], cycles, c["mg_cycles"], factor, st.iterations, c["iterations"]))
    assert abs(lam0 - c["re_lambda0"]) <= 0.1 * abs(c["re_lambda0"])
    assert cycles == c["mg_cycles"]
    assert st.status == helm.HELM_OK and st.rel_res <= P.tol
    assert abs(st.iterations - c["iterations"]) <= 0.25 * c["iterations"]
