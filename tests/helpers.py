"""Shared builders for the GPU tests: the same seeded problem goes to the CUDA path (through
the C-ABI binding) and to the CPU oracle."""
import math

import numpy as np


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def mg_params(helm, pc="csg", prec="c128", nu=(2, 2), omega=0.8, smoother="jacobi", gamma=(1, 1),
              coarsest_n=17, theta_a=math.pi / 14, beta=(-1.0, -0.5), re_lambda0=0.0, gs="fp64"):
    return helm.MGParams(kind=pc, theta_a=theta_a, beta1=beta[0], beta2=beta[1], re_lambda0=re_lambda0,
                         nu1=nu[0], nu2=nu[1], omega=omega, smoother=smoother, gamma_f=gamma[0],
                         gamma_c=gamma[1], coarsest_n=coarsest_n, prec=prec, gs=gs)


def gpu_handle(helm, P, **kw):
    """A handle for problem P (its grid, ECS, k^2; its CSG angle unless theta_a is given)."""
    import torch
    n = P.n if hasattr(P.n, "__len__") else [P.n] * P.dim
    kw.setdefault("theta_a", P.theta_a)
    k2 = torch.from_numpy(np.ascontiguousarray(P.k2)).cuda()
    mg = mg_params(helm, coarsest_n=kw.pop("coarsest_n", P.coarsest_n), **kw)
    r0lo, r0hi = P.layers
    return helm.helm_create(P.dim, n, k2, theta=P.theta, r0_lo=[r0lo] * P.dim, r0_hi=[r0hi] * P.dim,
                            lo=[P.lo] * P.dim, hi=[P.hi] * P.dim, mg=mg)


def oracle_pair(O, P, pc="csg", theta_a=None, beta=(-1.0, -0.5), re_lambda0=None):
    """The oracle's A and M for problem P (its CSG angle unless theta_a is given)."""
    theta_a = P.theta_a if theta_a is None else theta_a
    n = P.n if hasattr(P.n, "__len__") else [P.n] * P.dim
    z = [O.contour(n[a], P.lo, P.hi, P.theta, *P.layers) for a in range(P.dim)]
    return O.helmholtz_ops(z, P.k2, pc=pc, theta_a=theta_a, beta=beta, re_lambda0=re_lambda0)


def to_gpu(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t if dtype is None else t.to(dtype)


def to_np(t):
    return t.detach().cpu().numpy()


def small_problem_adjoint(n, kh=0.5):
    """A 2D well problem of n x n nodes for the adjoint checks (E = 2, growth toward the
    boundary up to k h = kh, Gaussian source of width 0.1)."""
    from paper_1012_4307_gb300 import workloads as W
    return W.Problem("adj", 2, n, W.k2_well_growth(2, n, E=2.0, kh_max=kh), W.gaussian_source(2, n, 0.1, 7),
                     coarsest_n=17)
