"""GB300-native constrained shortest paths on lattices (and general graphs of bounded
degree) by the water-flow cycle of I. Matic, arXiv 1511.06441.

The solver is the CUDA library ``libcsp.so`` (``csrc/``), reached through the C ABI
declared in ``include/csp.h``; :mod:`.csp` is the thin ctypes binding and
:mod:`.synth` generates seeded inputs.  Submodules load lazily so that the input
generator can be used without a GPU.
"""
__all__ = ["csp", "synth"]
