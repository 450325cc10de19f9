"""Re(lambda0) for the QD preconditioner (Section 5; Section 6's closing remark: from a
one-dimensional counterpart, or minus the largest discrete k^2), computed on the host by the
library's helm_qd_lambda0 (no GPU needed), pinned against dense eigenvalues of the oracle's
operators (numpy) and against the value printed in Table 1."""
import math

import numpy as np
import pytest

from paper_1012_4307_gb300 import workloads as W


@pytest.fixture(scope="module")
def helm():
    from paper_1012_4307_gb300 import helm as H
    H.load()
    return H


def dense_min_real(O, z_axes, k2):
    A = O.Op(z_axes, k2, a=1.0, bk=-1.0, c=0.0)
    return float(np.linalg.eigvals(A.dense()).real.min())


def problem_axes(P):
    return dict(dim=2, n=[P.n, P.n], theta=P.theta, r0_lo=[P.layers[0]] * 2, r0_hi=[P.layers[1]] * 2,
                lo=[P.lo] * 2, hi=[P.hi] * 2)


@pytest.mark.parametrize("builder", [
    lambda: W.paper_mp1(k=40.0, interior_cells=64, layer_cells=16),
    lambda: W.paper_mp2(k=4.0, nu=7.0, size=12.5, interior_cells=128, layer_cells=32),
    lambda: W.paper_mp3(k=2.0, size=12.5, interior_cells=128, layer_cells=32),
], ids=["mp1", "mp2", "mp3"])
def test_axis_counterpart_equals_dense_1d_eigenvalues(helm, oracle, builder):
    """Each axis's term is the smallest real part of the dense 1D operator's eigenvalues."""
    P = builder()
    prof = P.extra["k2_axis"]
    geo = problem_axes(P)
    got = helm.helm_qd_lambda0(k2_axis=prof, **geo)
    z = oracle.contour(P.n, P.lo, P.hi, P.theta, *P.layers)
    ref = sum(dense_min_real(oracle, [z], prof[a]) for a in range(2))
    assert abs(got - ref) <= 1e-9 * abs(ref), (got, ref)


def test_kronecker_sum_is_the_2d_eigenvalue(helm, oracle):
    """For a separable k^2 the sum of the axes' values is the smallest real part over the dense
    2D operator's eigenvalues (two different profiles, one-sided layer on one axis)."""
    n = 25
    x = np.linspace(0.0, 3.0, n)
    y = np.linspace(-1.5, 1.5, n)
    kx = 6.0 + 4.0 * np.exp(-(x - 1.0) ** 2)
    ky = 3.0 + 2.0 * np.cos(y)
    k2 = ky[:, None] + kx[None, :]
    r0lo, r0hi = [-1.0, -1.0], [2.2, 1.0]
    got = helm.helm_qd_lambda0(2, [n, n], [kx, ky], theta=math.pi / 6, r0_lo=r0lo, r0_hi=r0hi,
                               lo=[0.0, -1.5], hi=[3.0, 1.5])
    z = [oracle.contour(n, 0.0, 3.0, math.pi / 6, r0lo[0], r0hi[0]),
         oracle.contour(n, -1.5, 1.5, math.pi / 6, r0lo[1], r0hi[1])]
    ref = dense_min_real(oracle, z, k2)
    assert abs(got - ref) <= 1e-9 * abs(ref), (got, ref)


def test_max_k2_mode(helm):
    n = 33
    kx = np.linspace(1.0, 5.0, n)
    ky = np.linspace(2.0, 0.0, n)
    got = helm.helm_qd_lambda0(2, [n, n], [kx, ky], mode="max_k2")
    # interior nodes only: node 1 .. n-2 of each axis
    assert got == pytest.approx(-(kx[1:-1].max() + ky[1:-1].max()), rel=1e-15)


def test_table1_value(helm):
    """MP1 (k = 160, 256 + 2 x 64 cells, ECS pi/6): the one-dimensional counterpart gives the
    Re(lambda0) that Table 1 prints to two digits, -2.6e4."""
    P = W.paper_mp1(k=160.0)
    got = helm.helm_qd_lambda0(k2_axis=P.extra["k2_axis"], **problem_axes(P))
    assert round(got, -3) == -2.6e4 and -160.0 ** 2 < got < -160.0 ** 2 + 50.0, got


def test_rejects_bad_arguments(helm):
    with pytest.raises(helm.HelmError) as e:
        helm.helm_qd_lambda0(2, [17, 17], [np.zeros(17), np.zeros(17)], mode="max_k2", lo=[1.0, 1.0], hi=[0.0, 0.0])
    assert e.value.status == helm.HELM_ERR_ARG
    bad = np.zeros(17)
    bad[5] = np.nan
    with pytest.raises(helm.HelmError) as e:
        helm.helm_qd_lambda0(2, [17, 17], [bad, np.zeros(17)])
    assert e.value.status == helm.HELM_ERR_NONFINITE
