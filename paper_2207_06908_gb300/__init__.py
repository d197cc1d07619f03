"""GB300 (sm_103a) FDTD hot path of the elecode method (arXiv 2207.06908):
lossy-media Yee leapfrog with thin wires, CPML, current sources and probes.

Importing the package loads nothing; ``paper_2207_06908_gb300.fdtd`` loads the
CUDA library on first use and fails loudly when it is missing.
"""
__all__ = ["fdtd", "workloads"]
