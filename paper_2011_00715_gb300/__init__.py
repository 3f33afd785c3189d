"""GB300-native Jacobi-preconditioned conjugate-gradient solve over CSR
matrices (the PETSc GPU solve loop of arXiv 2011.00715: MatMult, PCApply
Jacobi, VecAXPY/VecAYPX/VecDot/VecNorm), in hand-written CUDA for sm_103a
behind a C ABI (include/gbs.h).

``gbs`` is the Python binding of that ABI; ``inputs`` holds the seeded
synthetic problem generators; ``build`` compiles the library in-tree.
"""
__all__ = ["gbs", "inputs", "build"]
