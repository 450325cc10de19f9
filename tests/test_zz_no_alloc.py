"""The allocation-free entry point helm_mg_conv_noalloc against the allocating helm_mg_conv.

helm_mg_conv allocates its work area with cudaMalloc on first use; callers that cannot
allocate at the point of the call (for example during CUDA graph capture, or under a fixed
device-memory budget) use helm_mg_conv_noalloc, which keeps its work vectors in one fixed
device array.  Both run the same kernels, so their results must agree to rounding, call after
call, although the array keeps the previous call's contents.

This file is collected last, so that a stopped-at-first-failure run has already run every
other test; it also passes when run alone in a fresh process.
"""
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


@pytest.mark.parametrize("dim,n,prec", [(2, 65, "c128"), (2, 129, "c64"), (3, 17, "c128")])
def test_noalloc_matches_allocating_entry_point(helm, dim, n, prec):
    P = W.Problem("t", dim, n, W.k2_well_growth(dim, n, kh_max=0.3), W.gaussian_source(dim, n, 0.1, 3),
                  coarsest_n=17 if dim == 2 else 9)
    h = gpu_handle(helm, P, pc="csl", prec=prec)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    b = to_gpu(P.f).to(dt)
    x_ref, n_ref, f_ref = helm.helm_mg_conv(h, b, tol=1e-6, maxcyc=60)
    tol = 1e-12 if prec == "c128" else 1e-5
    for call in range(2):
        x = torch.zeros_like(b)
        ncyc, fac = helm.helm_mg_conv_noalloc(h, b, x, tol=1e-6, maxcyc=60)
        assert ncyc == n_ref
        assert abs(fac - f_ref) <= tol * max(abs(f_ref), 1e-30)
        err = float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref))
        assert err <= tol, (call, err)


def test_noalloc_rejects_grids_beyond_its_array(helm):
    n = 1025  # 1,050,625 nodes need ~32 MiB of scratch, beyond the 16 MiB array
    P = W.Problem("t", 2, n, W.k2_constant(2, n, 5.0), W.gaussian_source(2, n, 0.1, 1), coarsest_n=17)
    h = gpu_handle(helm, P, pc="csl", prec="c64")
    b = to_gpu(P.f).to(torch.complex64)
    x = torch.zeros_like(b)
    with pytest.raises(helm.HelmError) as e:
        helm.helm_mg_conv_noalloc(h, b, x, maxcyc=2)
    assert e.value.status == helm.HELM_ERR_ARG and "scratch" in str(e.value)
    assert float(x.abs().max()) == 0.0
