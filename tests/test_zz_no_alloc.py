"""The allocation-free entry point helm_mg_conv_noalloc against the allocating helm_mg_conv.

helm_mg_conv allocates its work area with cudaMalloc on first use.  Callers that cannot
allocate at the point of the call (a service whose device memory is sized once at start-up, or
a loop that cannot afford the device-wide synchronisation an allocation may cause) use
helm_mg_conv_noalloc, which keeps its work vectors in one fixed device array.  Both run the
same kernels, so their results must agree to rounding, call after call, although the array
keeps the previous call's contents; and the allocation-free calls must not take any device
memory.

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


def problem(dim, n):
    return W.Problem("t", dim, n, W.k2_well_growth(dim, n, kh_max=0.3), W.gaussian_source(dim, n, 0.1, 3),
                     coarsest_n=17 if dim == 2 else 9)


def test_noalloc_takes_no_device_memory(helm):
    """On a fresh 513 x 513 handle (whose Krylov workspace, were it allocated, would take about
    13 MB), two allocation-free calls leave the device's free memory where it was.  A first call
    on another handle of the same grid does the one-time set-up before the measurement: loading
    the library's device code on first launch (which also places the fixed array) and looking
    up the array's address."""
    P = problem(2, 513)
    b = to_gpu(P.f).to(torch.complex64)
    hw = gpu_handle(helm, P, pc="csl", prec="c64")
    helm.helm_mg_conv_noalloc(hw, b, torch.zeros_like(b), tol=1e-6, maxcyc=3)
    h = gpu_handle(helm, P, pc="csl", prec="c64")
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        ncyc, fac = helm.helm_mg_conv_noalloc(h, b, x, tol=1e-6, maxcyc=40)
        assert ncyc >= 1 and np.isfinite(fac)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)
    # the allocating entry point on the same handle does take memory (its Krylov workspace),
    # so the measurement above can see an allocation of this size
    x_ref, n_ref, _ = helm.helm_mg_conv(h, b, tol=1e-6, maxcyc=40)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 < free1, (free1, free2)
    assert ncyc == n_ref
    err = float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref))
    assert err <= 1e-5


@pytest.mark.parametrize("dim,n,prec", [(2, 65, "c128"), (2, 129, "c64"), (3, 17, "c128")])
def test_noalloc_matches_allocating_entry_point(helm, dim, n, prec):
    P = problem(dim, n)
    h = gpu_handle(helm, P, pc="csl", prec=prec)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    b = to_gpu(P.f).to(dt)
    tol = 1e-12 if prec == "c128" else 1e-5
    # the allocation-free calls first, on the fresh handle, then the allocating reference
    outs = []
    for call in range(2):
        x = torch.zeros_like(b)
        outs.append((x,) + helm.helm_mg_conv_noalloc(h, b, x, tol=1e-6, maxcyc=60))
    x_ref, n_ref, f_ref = helm.helm_mg_conv(h, b, tol=1e-6, maxcyc=60)
    for call, (x, ncyc, fac) in enumerate(outs):
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
