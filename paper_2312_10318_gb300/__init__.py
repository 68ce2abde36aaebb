"""GB300-native D2Q9 TRT-RLB lattice Boltzmann library (arXiv 2312.10318).

The fused stream-and-collide step runs in hand-written CUDA for sm_103a inside
``libtrtrlb.so`` (C ABI: ``include/trtrlb.h``).  This package is its Python
binding plus host-side helpers: parameter mapping, seeded workloads, the
serving loop and the autotuner.  Importing the package does not load the
library; constructing a Lattice does, and fails loudly if it is not built.
"""
from __future__ import annotations

__all__ = ["Lattice", "Slabs", "params", "workloads"]


def __getattr__(name):
    if name in ("Lattice", "Slabs"):
        from . import lattice
        return getattr(lattice, name)
    if name in ("params", "workloads"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
