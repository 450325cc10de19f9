"""GB300-native matrix-free ECS Helmholtz solver (bin Zubair, Reps & Vanroose, arXiv 1012.4307).

The compute path is the C-ABI library ``libhelm.so`` (hand-written sm_103a CUDA kernels); the
Python binding in :mod:`paper_1012_4307_gb300.helm` only marshals arguments.  Submodules are
imported lazily so that the seeded input generators can be used without a GPU.
"""
__all__ = ["helm", "workloads"]
