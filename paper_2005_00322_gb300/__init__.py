"""GB300-native DTT-based PSTD (sine/cosine pseudospectral time domain) solver.

The compute path is the CUDA library libpstd.so (C ABI in include/pstd.h);
``Solver`` is a thin binding that marshals torch device tensors into it.
Importing the package does not load the library; constructing a ``Solver``
does, and fails loudly if it is not built or no GPU is present.
"""

__all__ = ["Solver", "inputs"]


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    raise AttributeError(name)
