"""GB300 (sm_103a) HSDE-ADMM for chordally sparse SDPs.

The compute path is libhsde.so (CUDA kernels behind the C-ABI of
include/hsde.h); ``paper_1611_01828_gb300.hsde`` is its ctypes binding.
Importing the binding raises if the library has not been built: there is no
CPU fallback.
"""
import importlib

__all__ = ["hsde"]


def __getattr__(name):
    if name in ("hsde",):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
