"""GB300 (sm_103a) tangent-point energy and H^s Sobolev descent (Repulsive Curves, arXiv 2006.07859).

The compute path is the C-ABI CUDA library ``libtpe.so`` built from ``csrc/``; ``tpe.py`` is a thin
ctypes binding with the same entry-point names.  PyTorch supplies device memory and streams only.
"""
from .tpe import *  # noqa: F401,F403
