"""GB300 baryon pasting (Osato & Nagai, arXiv:2201.02632): the per-halo ICM solve,
particle-based pasting (PP) and halo-based pasting (HP) on one GPU.

The computation lives in libbp.so (hand-written sm_103a CUDA behind the C ABI of
include/bp.h).  This package holds the ctypes binding (``api``), the in-tree
build (``build``) and the seeded synthetic workloads (``inputs``).  PyTorch is
used only for device memory and streams.
"""
from __future__ import annotations

__all__ = ["api", "build", "inputs"]


def __getattr__(name):
    if name in ("api", "build", "inputs"):
        import importlib

        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
