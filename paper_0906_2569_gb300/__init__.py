"""Plane-wave H|psi> and block-Davidson eigensolver on one GB300 (sm_103a).

The compute path is libhpsi.so (CUDA kernels behind a C ABI, include/hpsi.h); ``binding`` is its
ctypes binding with the same function names, ``build`` compiles it in-tree with nvcc.
"""
from . import binding  # noqa: F401

__all__ = ["binding"]
