"""Writes oracle_iterations.json: iterations and wall time of the CPU oracle's FP64 FGMRES(30)
(CSG preconditioner, one V(2,2) omega-Jacobi cycle, omega 0.8) on the 2D 1025 x 1025 well
problem to a relative residual of 1e-8.  Calls only oracle/ and the seeded input generators.
The benchmark's CPU baseline times a few oracle iterations and scales by this count."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1012_4307_gb300 import workloads as W  # noqa: E402


def main(n=1025):
    P = W.config_2d_well(n)
    z = O.axes(2, P.n, theta=P.theta, r0lo=-P.r0, r0hi=P.r0)
    A, M = O.helmholtz_ops(z, P.k2, pc="csg", theta_a=P.theta_a)
    t0 = time.time()
    mg = O.MG(M, P.coarsest_n, P.nu1, P.nu2, P.omega, P.smoother)
    x, st = O.fgmres(A, mg, P.f, tol=1e-8, restart=30, maxit=2000)
    dt = time.time() - t0
    out = {"workload": P.name, "unknowns": P.unknowns, "tol": 1e-8, "restart": 30,
           "iterations": st["iterations"], "restarts": st["restarts"], "rel_res": st["rel_res"],
           "status": st["status"], "seconds": dt, "threads": 1}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")
    with open(path, "w") as fh:
        json.dump({P.name: out}, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1025)
