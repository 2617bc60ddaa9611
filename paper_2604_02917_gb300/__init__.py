"""GB300 (sm_103a) NPGA library for constrained mean--variance portfolios.

The compute path lives in ``libmv.so`` (hand-written CUDA behind the C ABI of
``include/mv.h``).  ``paper_2604_02917_gb300.mv`` is a thin ctypes binding
with the same names; it only marshals arguments (PyTorch supplies device
memory and streams).  Importing this package does not load the library; the
first call into ``mv`` does, and fails loudly if it was not built.
"""

__all__ = ["mv"]
