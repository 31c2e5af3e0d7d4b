"""B300-native (sm_103a) ExpRK22 / WENO5 / FFT propagator for the KZK-type
sonic-boom equation of Einkemmer, Ostermann & Residori (arXiv:2103.06080).

The computation lives in ``libkzk.so`` (C ABI in ``include/kzk.h``); this
package holds the ctypes binding (``_lib``), a thin Plan wrapper (``api``),
the autograd wrapper (``autograd``) and the seeded input generators
(``inputs``).  Submodules are imported lazily so that ``inputs`` can be used
without loading the CUDA library.
"""
__all__ = ["api", "inputs", "autograd"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
