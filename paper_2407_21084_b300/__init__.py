"""B300 (sm_103a) implementation of the QRMC Picard iteration of Gobet,
Lopez-Salas and Vazquez (arXiv 2407.21084).

The arithmetic lives in libqrmc.so (hand-written CUDA behind the C-ABI of
include/qr.h); ``Solver`` is a thin ctypes binding. Importing this package
does not load the library; the first Solver (or ``load()``) does, and raises
if it is missing: there is no CPU fallback.
"""
from . import workloads  # noqa: F401  (no arithmetic, no library load)


def load():
    from . import _lib

    return _lib.load()


def __getattr__(name):
    if name in ("Solver", "philox_words", "sample"):
        from . import solver

        return getattr(solver, name)
    raise AttributeError(name)
