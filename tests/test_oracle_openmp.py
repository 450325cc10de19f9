"""The all-cores build of the oracle (-fopenmp, used only for the CPU baseline) computes exactly
what the single-threaded build computes: only loops whose iterations are independent are shared
out, so an FGMRES solve with its multigrid preconditioner and a Bi-CGSTAB solve give
bit-identical iterates, residual histories and iteration counts."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, %r)
from oracle import oracle as O
from paper_1012_4307_gb300 import workloads as W
P = W.config_small(33)
A, M = O.helmholtz_ops(O.axes(2, P.n), P.k2, pc="csg")
mg = O.MG(M, 17, 2, 2, 0.8)
x, st = O.fgmres(A, mg, P.f, tol=1e-10, restart=30, maxit=200, history=True)
y, st2 = O.bicgstab(A, mg, P.f, tol=1e-10, maxit=200)
np.save(sys.argv[1], np.stack([x, y]))
print(json.dumps({"it": st["iterations"], "it2": st2["iterations"], "hist": st["history"].tolist(),
                  "threads": O.threads()}))
'''


def run(tmp_path, openmp):
    env = dict(os.environ, HELM_ORACLE_OPENMP="1" if openmp else "0", OMP_NUM_THREADS="4")
    out = str(tmp_path / ("omp.npy" if openmp else "ser.npy"))
    r = subprocess.run([sys.executable, "-c", CHILD % ROOT, out], env=env, capture_output=True, text=True,
                       check=True)
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(out)


def test_openmp_build_is_bit_identical(tmp_path, oracle):
    meta_s, xs = run(tmp_path, False)
    meta_p, xp = run(tmp_path, True)
    assert meta_s["threads"] == 1 and meta_p["threads"] == 4
    assert meta_s["it"] == meta_p["it"] and meta_s["it2"] == meta_p["it2"]
    assert meta_s["hist"] == meta_p["hist"]
    assert np.array_equal(xs, xp)
