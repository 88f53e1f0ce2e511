"""Tersoff many-body potential on one GB300: energy/force hot path (Algorithm 1
of Hoehnerbach, Ismail & Bientinesi), cell-list/Verlet neighbour build, velocity
Verlet, and a continuous-batching MD server, all behind the C-ABI library
``libtersoff.so`` (declared in ``include/tersoff.h``).

Importing the package is cheap; the ctypes binding to the CUDA library lives in
``paper_1710_00882_gb300.tersoff`` and fails loudly when the library is missing.
"""
__all__ = ["workloads", "params", "tersoff"]
