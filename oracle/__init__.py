"""Plain FP64 CPU oracle for the asymptotic parareal method (1D rotating shallow water).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or executes anything here, and
this package imports nothing from the product path.
"""
from .rsw import *  # noqa: F401,F403
